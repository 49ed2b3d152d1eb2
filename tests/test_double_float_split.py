"""The integer split of an FP64 value into a pair of FP32 values (hi + lo) and
the widening back, as the double-float sine transforms do them on the IEEE 754
encodings, restated with numpy bit operations and checked against exact
arithmetic: hi is the value rounded to 24 significant bits, lo the rest
rounded to FP32, |lo| <= ulp(hi) / 2, and hi + lo equals the value within
2^-48 of it over the FP32 exponent range (within one subnormal ulp, 2^-149,
where lo falls into the FP32 subnormals and is rounded twice); below 2^-126
the pair is zero, values that round to 2^128 or more give an infinite hi.
The split also takes an exact power-of-two scaling 2^eshift, added to the
exponent of finite nonzero values."""
import numpy as np
import pytest


def f32(bits):
    return np.array(bits, dtype=np.uint32).view(np.float32)


def split(x, eshift=0):
    b = np.array(x, dtype=np.float64).view(np.uint64)
    h32 = (b >> np.uint64(32)).astype(np.uint32)
    l32 = (b & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    E = int((h32 >> np.uint32(20)) & np.uint32(0x7FF))
    if E != 0 and E != 2047:
        E += eshift
    sign = h32 & np.uint32(0x80000000)
    if E < 897:
        return f32(sign), np.float32(0.0)
    if E > 1150:
        nan = E == 2047 and ((int(h32) & 0xFFFFF) | int(l32)) != 0
        return f32(sign | np.uint32(0x7FC00000 if nan else 0x7F800000)), np.float32(0.0)
    m23 = ((int(h32) & 0xFFFFF) << 3) | (int(l32) >> 29)
    rem = int(l32) & 0x1FFFFFFF
    up = rem >> 28
    hi = f32(np.uint32(((int(sign) | ((E - 896) << 23) | m23) + up) & 0xFFFFFFFF))
    r = rem - (up << 29)
    m = abs(r)
    mh = np.float32(f32(np.uint32(0x4B000000 | (m >> 14))) - np.float32(8388608.0))
    ml = np.float32(f32(np.uint32(0x4B000000 | (m & 0x3FFF))) - np.float32(8388608.0))
    small = E < 949
    scale = f32(np.uint32(((E - 884) if small else (E - 948)) << 23))
    post = np.float32(2.0 ** -64) if small else np.float32(1.0)
    # one rounding for mh 2^14 + ml (the FMA), an exact power-of-two scaling (normal range),
    # and for small E a second rounding by 2^-64 into the subnormals
    lo = np.float32(np.float32(np.float64(mh) * 16384.0 + np.float64(ml)) * scale) * post
    return hi, (-lo if ((r < 0) != (int(sign) != 0)) else lo)


def widen(f):
    u = int(np.array(f, dtype=np.float32).view(np.uint32))
    e = (u >> 23) & 0xFF
    sign = u & 0x80000000
    m = u & 0x7FFFFF
    if e == 0:
        hi32, lo32 = sign, 0
    elif e == 0xFF:
        hi32, lo32 = sign | 0x7FF00000 | (0x80000 if m else 0), 0
    else:
        hi32, lo32 = sign | ((e + 896) << 20) | (m >> 3), (m << 29) & 0xFFFFFFFF
    return np.array((hi32 << 32) | lo32, dtype=np.uint64).view(np.float64)[()]


def test_split_is_accurate_and_normalised_over_the_fp32_range():
    rng = np.random.default_rng(3)
    for _ in range(20000):
        x = float(rng.choice([-1, 1]) * 2.0 ** rng.integers(-100, 120) * rng.uniform(1, 2))
        hi, lo = split(x)
        assert np.float64(hi) + np.float64(lo) == pytest.approx(x, rel=2.0 ** -48, abs=0)
        ulp = np.spacing(np.abs(hi))
        assert abs(lo) <= 0.5 * ulp * (1 + 2.0 ** -20)
        assert np.float32(hi) == np.float32(x) or abs(np.float64(hi) - x) <= ulp   # hi is x to 24 bits


def test_split_edges_and_widening():
    assert split(0.0) == (0.0, 0.0) and np.signbit(split(-0.0)[0])
    assert split(1e-39)[0] == 0.0                      # below the FP32 normal range
    assert np.isinf(split(1e39)[0]) and np.isnan(split(float("nan"))[0])
    hi, lo = split(1.0 + 2.0 ** -30)
    assert hi == 1.0 and lo == np.float32(2.0 ** -30)
    for f in [1.5, -3.25e-20, 6.0e30, np.float32(1.1754944e-38)]:
        assert widen(np.float32(f)) == np.float64(np.float32(f))
    assert widen(np.float32(0.0)) == 0.0 and np.isinf(widen(np.float32("inf")))
    assert np.isnan(widen(np.float32("nan")))


def test_split_down_to_the_subnormal_lo_and_the_top_carry():
    """Exponents -126 ... 127: where lo lies below 2^-126 it is rounded twice (24
    bits, then into the subnormals) and the pair is within 2^-149 of x; an
    all-ones 23-bit fraction with the round bit set carries into the exponent,
    and at the top of the range into infinity."""
    rng = np.random.default_rng(4)
    for _ in range(20000):
        e = int(rng.integers(-126, 128))
        x = float(rng.choice([-1, 1]) * 2.0 ** e * rng.uniform(1, 2))
        hi, lo = split(x)
        if np.isinf(hi):
            assert abs(x) >= (2.0 - 2.0 ** -24) * 2.0 ** 127
            continue
        err = abs((np.float64(hi) + np.float64(lo)) - x)
        assert err <= max(2.0 ** -48 * abs(x), 2.0 ** -149), (x, err)
    for e in (-126, -120, -100, 0, 50, 126):
        x = (2.0 - 2.0 ** -25) * 2.0 ** e            # m23 all ones, round bit set
        hi, lo = split(x)
        assert np.float64(hi) == 2.0 ** (e + 1)
        assert abs((np.float64(hi) + np.float64(lo)) - x) <= max(2.0 ** -48 * x, 2.0 ** -149)
    hi, _ = split((2.0 - 2.0 ** -25) * 2.0 ** 127)    # rounds to 2^128: beyond FP32
    assert np.isinf(hi)


def test_split_with_a_power_of_two_scaling():
    """split(x, s) equals split(x 2^s) for data far outside the FP32 range brought
    into it, and keeps zero, infinity and NaN."""
    rng = np.random.default_rng(5)
    for _ in range(2000):
        s = int(rng.integers(-900, 900))
        x = float(rng.choice([-1, 1]) * 2.0 ** (-s + int(rng.integers(-60, 60))) * rng.uniform(1, 2))
        assert split(x, s) == split(x * 2.0 ** s)
    assert split(0.0, 300) == (0.0, 0.0)
    assert np.isinf(split(float("inf"), -500)[0]) and np.isnan(split(float("nan"), 7)[0])
    assert split(1e-300, 0)[0] == 0.0 and split(1e-300, 997)[0] != 0.0
