"""The FP64 -> FP32 hi/lo split, the centre-of-mass quotient of the
moments kernels and the grid quantisation's floor, restated on the CPU in
exact arithmetic and checked against their definitions: hi = RN32(v), lo =
RN32(v - hi) (numpy's float32 rounding), RN(S / M) (the correctly rounded
quotient of the exact rationals), and min(2^21 - 1, max(0, floor(u))).
CPU only."""
import struct
from fractions import Fraction

import numpy as np


def bits(v):
    return struct.unpack("<Q", struct.pack("<d", v))[0]


def f32bits(u):
    return struct.unpack("<f", struct.pack("<I", u))[0]


def split_int(v):
    """The kernels' integer split (None: the FP64 instructions take it)."""
    b = bits(v)
    e = (b >> 52) & 0x7FF
    if e < 949 or e > 1149:
        return None
    sig = (b & ((1 << 52) - 1)) | (1 << 52)
    keep = sig >> 29
    rem = sig & ((1 << 29) - 1)
    up = rem > (1 << 28) or (rem == (1 << 28) and (keep & 1))
    diff = rem - ((1 << 29) if up else 0)
    keep += 1 if up else 0
    eh = e - 1023 + 127
    if keep == 1 << 24:
        keep >>= 1
        eh += 1
    sgn = (b >> 63) << 31
    hi = f32bits(sgn | (eh << 23) | (keep & 0x7FFFFF))
    if diff == 0:
        return np.float32(hi), np.float32(0.0)
    f = np.float32(diff)  # one rounding, as the int-to-float conversion
    lo = np.float32(f * np.float32(2.0 ** (e - 1075)))  # exact power-of-two scale
    return np.float32(hi), np.float32(-lo if sgn else lo)


def test_integer_split_equals_fp64_definition():
    rng = np.random.default_rng(20261203)
    vals = list(rng.standard_normal(20000) * 10.0 ** rng.uniform(-30, 30, 20000))
    # halfway cases: the 29 dropped bits exactly 1 followed by zeros, both parities
    for _ in range(2000):
        sig = int(rng.integers(1 << 23, 1 << 24))
        e = int(rng.integers(-60, 60))
        vals.append(float(Fraction(sig * 2 + 1, 2) * Fraction(2) ** e) * (1 if rng.random() < 0.5 else -1))
    # values just below a power of two (rounding carries into the exponent)
    vals += [np.nextafter(2.0 ** k, 0.0) for k in range(-100, 100)]
    vals += [0.0, -0.0, 1.0, -1.0, 2.0 ** -126, 2.0 ** 127, 1e-300, 1e300]
    taken = 0
    for v in vals:
        r = split_int(float(v))
        if r is None:
            continue
        taken += 1
        hi = np.float32(v)
        lo = np.float32(float(v) - float(hi))
        assert r[0].tobytes() == hi.tobytes(), v
        assert r[1].tobytes() == lo.tobytes(), v
    assert taken > 15000


def test_integer_split_with_wrong_rounding_is_caught():
    """Planted mistake: rounding halfway cases up instead of to even."""
    v = float(Fraction((1 << 23) * 2 + 1, 2))  # 2^23 + 1/2: a halfway case with an even keep
    b = bits(v)
    sig = (b & ((1 << 52) - 1)) | (1 << 52)
    keep_wrong = (sig >> 29) + 1
    assert keep_wrong & 0x7FFFFF != split_int(v)[0].view(np.uint32) & 0x7FFFFF


def markstein(S, M):
    y = float(Fraction(1) / Fraction(M))                 # RN(1/M)
    q0 = float(Fraction(S) * Fraction(y))                # RN(S y)
    r = float(Fraction(S) - Fraction(M) * Fraction(q0))  # RN(S - M q0), one fused multiply-add
    return float(Fraction(q0) + Fraction(r) * Fraction(y))   # RN(q0 + r y), one fused multiply-add


def test_markstein_quotient_equals_correctly_rounded_division():
    rng = np.random.default_rng(1990)
    cases = []
    for _ in range(20000):
        M = float(rng.uniform(1.0, 2.0)) * 2.0 ** int(rng.integers(-60, 60))
        S = float(rng.standard_normal()) * 2.0 ** int(rng.integers(-60, 60))
        cases.append((S, M))
    # all-ones significands, exact multiples, masses summed from equal parts
    for k in range(200):
        M = float(np.nextafter(2.0 ** (k % 40 - 20), np.inf)) if k % 2 else float(np.nextafter(2.0 ** (k % 40 - 19), 0.0))
        cases.append((M * float(rng.integers(-10 ** 6, 10 ** 6)), M))
        m = 1.0 / 3.0
        Msum = 0.0
        for _ in range(k % 16 + 1):
            Msum += m
        cases.append((Msum * 0.7, Msum))
    for S, M in cases:
        assert markstein(S, M) == float(Fraction(S) / Fraction(M)), (S, M)


def test_quotient_without_the_correction_step_is_caught():
    """Planted mistake: q0 = RN(S RN(1/M)) alone is not always RN(S / M)."""
    rng = np.random.default_rng(7)
    wrong = 0
    for _ in range(5000):
        M = float(rng.uniform(1.0, 2.0))
        S = float(rng.uniform(1.0, 2.0))
        y = float(Fraction(1) / Fraction(M))
        q0 = float(Fraction(S) * Fraction(y))
        wrong += q0 != float(Fraction(S) / Fraction(M))
    assert wrong > 0


QMAX = (1 << 21) - 1


def floor_bits(u):
    """The kernels' clamped floor of u from its bits (integer operations)."""
    b = bits(u)
    if b >= 1 << 63 or b == 0:  # negative (sign bit set) or +0
        return 0
    e = b >> 52
    if e < 1023:
        return 0
    if e >= 1023 + 21:
        return QMAX
    m = (b & ((1 << 52) - 1)) | (1 << 52)
    return m >> (52 - (e - 1023))


def test_quantisation_floor_from_bits_equals_clamped_floor():
    rng = np.random.default_rng(1601)
    vals = [0.0, -0.0, 5e-324, 1e-300, 0.5, 1.0, np.nextafter(1.0, 0.0), np.nextafter(1.0, 2.0),
            float(QMAX), np.nextafter(float(QMAX), 0.0), float(QMAX) + 0.5, np.nextafter(2.0 ** 21, 0.0),
            2.0 ** 21, 2.0 ** 21 + 1.0, 1e300, float("inf"), -1.0, -1e-300, -2.0 ** 22]
    ints = rng.integers(0, 1 << 21, 2000).astype(float)
    vals += list(ints) + [np.nextafter(v, 0.0) for v in ints] + [np.nextafter(v, np.inf) for v in ints]
    vals += list(rng.uniform(-10.0, 2.0 ** 21 + 10.0, 4000)) + list(2.0 ** rng.uniform(-60, 30, 2000))
    for u in vals:
        want = 0 if u < 1.0 else (QMAX if u >= 2.0 ** 21 else int(Fraction(u)) // 1)
        assert floor_bits(float(u)) == want, u


def test_quantisation_floor_planted_mistake_is_caught():
    """An off-by-one shift (the exponent bias taken as 1022) fails the
    definition: the check is not vacuous."""
    def wrong(u):
        b = bits(u)
        if b >= 1 << 63 or b == 0:
            return 0
        e = b >> 52
        if e < 1023:
            return 0
        if e >= 1023 + 21:
            return QMAX
        m = (b & ((1 << 52) - 1)) | (1 << 52)
        return m >> (52 - (e - 1022))
    assert any(wrong(u) != min(QMAX, int(u)) for u in (1.0, 3.5, 1000.25))
