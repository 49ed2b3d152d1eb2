"""The integer split of an FP64 value into a pair of FP32 values (hi + lo) and
the widening back, as the double-float sine transforms do them on the IEEE 754
encodings, restated with numpy bit operations and checked against exact
arithmetic: hi is the value rounded to 24 significant bits, lo the rest
rounded to FP32, |lo| <= ulp(hi) / 2, and hi + lo equals the value within
2^-48 of it over the FP32 exponent range; below 2^-126 the pair is zero, from
2^128 on hi is infinite."""
import numpy as np
import pytest


def f32(bits):
    return np.array(bits, dtype=np.uint32).view(np.float32)


def split(x):
    b = np.array(x, dtype=np.float64).view(np.uint64)
    h32 = (b >> np.uint64(32)).astype(np.uint32)
    l32 = (b & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    E = ((h32 >> np.uint32(20)) & np.uint32(0x7FF)).astype(np.int64)
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
    # one rounding for mh 2^14 + ml (the FMA), then exact power-of-two scalings (normal range)
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
