"""The arithmetic of the tensor-core sine transform, restated in exact integers on the CPU.

The kernel (csrc/stmg_tc.cuh) writes a line x scaled by its largest exponent as 56-bit integers
F = |x| 2^(1078 - E) split into eight 7-bit digits, S/2 (S_jk = sin(pi j k / Nf)) as eight
balanced base-128 digits in [-64, 64], sums the digit products of weight g = s + t <= 7 over K
into one FP32 accumulator per g, and rounds W = sum_g C_g 2^(7 (7 - g)) once to FP64.  These
tests check, without a GPU, the two facts the design rests on: every partial sum of an
accumulator stays below 2^24 (so FP32 holds it exactly) for Nf <= 256 and not for Nf = 512, and
the dropped pairs and the truncation keep the result within 5e-16 of sqrt(Nf/2) ||x||_2.
"""
from fractions import Fraction
import math

import numpy as np
import pytest

mp = pytest.importorskip("mpmath").mp


def sine_digits(Nf):
    """e[t][k][m]: balanced base-128 digits of S/2, most significant first (as the host table)."""
    mp.dps = 40
    e = np.zeros((8, Nf, Nf), dtype=np.int64)
    for k in range(Nf):
        for m in range(Nf):
            v = mp.sin(mp.pi * ((k * m) % (2 * Nf)) / Nf) / 2
            for t in range(8):
                v *= 128
                d = int(mp.nint(v))
                v -= d
                e[t, k, m] = d
    return e


def line_digits(x):
    """Digits d[s][k] of F_k = |x_k| 2^(1078 - E) (E the largest exponent of the line), signs."""
    xs = np.concatenate([[0.0], x])           # slot k = 0 is zero
    E = max((math.frexp(v)[1] + 1022 for v in xs if v != 0.0), default=None)
    d = np.zeros((8, xs.size), dtype=np.int64)
    sgn = np.where(xs < 0, -1, 1)
    if E is None:
        return d, sgn, 0
    for k, v in enumerate(xs):
        if v == 0.0:
            continue
        F = int(Fraction(abs(v)) * Fraction(2) ** (1078 - E))   # truncated, < 2^56
        assert F < 2 ** 56
        for s in range(8):
            d[s, k] = (F >> (7 * (7 - s))) & 127
    return d, sgn, E


def model_transform(x, e):
    """y_m = 2 * 2^(E - 1085) sum_g C_g 2^(7 (7 - g)) with the kernel's pairs; returns (y, max |partial sum|)."""
    Nf = e.shape[1]
    d, sgn, E = line_digits(x)
    if E == 0:
        return np.zeros(Nf - 1), 0
    sd = d * sgn                               # signed digits
    C = np.zeros((8, Nf), dtype=np.int64)
    worst = 0
    for g in range(8):
        for s in range(g + 1):
            t = g - s
            # accumulate K in chunks of 16 as the MMAs do; track the largest running sum
            for k0 in range(0, Nf, 16):
                C[g] += sd[s, k0:k0 + 16] @ e[t, k0:k0 + 16, :]
                worst = max(worst, int(np.abs(C[g]).max()))
    W = [sum(int(C[g, m]) << (7 * (7 - g)) for g in range(8)) for m in range(1, Nf)]
    y = np.array([float(Fraction(w) * Fraction(2) ** (E - 1084)) for w in W])   # one rounding
    return y, worst


def exact_transform(x, Nf):
    mp.dps = 40
    return np.array([float(sum(mp.mpf(float(x[j - 1])) * mp.sin(mp.pi * ((j * m) % (2 * Nf)) / Nf)
                               for j in range(1, Nf))) for m in range(1, Nf)])


def line_scale(x, Nf):
    """sqrt(Nf / 2) ||x||_2 without underflow or overflow (x scaled by its largest power of two)."""
    m = float(np.max(np.abs(x)))
    if m == 0.0:
        return 0.0
    e = math.frexp(m)[1]
    return math.sqrt(Nf / 2) * math.ldexp(float(np.linalg.norm(np.ldexp(x, -e))), e)


def test_accumulator_bound_holds_up_to_256_and_fails_at_512():
    """|C_g| <= (Nf - 1) * 127 * 64 * (g + 1): below 2^24 for Nf = 256 at g = 7, above for Nf = 512."""
    bound = lambda Nf, g: (Nf - 1) * 127 * 64 * (g + 1)
    assert max(bound(256, g) for g in range(8)) < 2 ** 24
    assert bound(512, 7) >= 2 ** 24
    # the digit ranges behind the bound: data digits in [0, 127], sine digits in [-64, 64]
    e = sine_digits(64)
    assert int(np.abs(e).max()) <= 64


@pytest.mark.parametrize("Nf,seed", [(64, 0), (64, 1)])
def test_model_matches_exact_sums(Nf, seed):
    e = sine_digits(Nf)
    rng = np.random.default_rng(seed)
    n = Nf - 1
    lines = [rng.uniform(-1, 1, n) * 2.0 ** rng.integers(-30, 30),
             np.where(np.arange(n) % 2 == 0, rng.uniform(-1, 1, n) * 1e12, rng.uniform(-1, 1, n) * 1e-12),
             np.ldexp(rng.uniform(-1, 1, n), -1040),          # subnormal line
             np.zeros(n)]
    for x in lines:
        y, worst = model_transform(x, e)
        assert worst < 2 ** 24                                # every FP32 partial sum exact
        ref = exact_transform(x, Nf)
        scale = line_scale(x, Nf)
        if scale == 0.0:
            assert np.all(y == 0.0)
            continue
        err = np.abs(y - ref) - 2.0 ** -1074                  # the subnormal grid cannot do better
        assert float(np.max(np.maximum(err, 0.0))) / scale < 5e-16


def test_model_catches_a_dropped_digit_pair():
    """Leaving out the weight-7 pairs (the last ones the kernel keeps) breaks the 5e-16 bound of
    test_model_matches_exact_sums (measured about 1.3e-15), so that bound would notice a kernel that
    stopped one weight early; the pairs of weight 8 and above, which the kernel drops, are 128 times
    smaller again."""
    Nf = 64
    e = sine_digits(Nf)
    x = np.random.default_rng(3).uniform(-1, 1, Nf - 1)
    d, sgn, E = line_digits(x)
    sd = d * sgn
    C = np.zeros((8, Nf), dtype=np.int64)
    for g in range(7):                                       # g = 7 dropped
        for s in range(g + 1):
            C[g] += sd[s] @ e[g - s]
    W = [sum(int(C[g, m]) << (7 * (7 - g)) for g in range(8)) for m in range(1, Nf)]
    y = np.array([float(Fraction(w) * Fraction(2) ** (E - 1084)) for w in W])
    ref = exact_transform(x, Nf)
    scale = line_scale(x, Nf)
    assert float(np.max(np.abs(y - ref))) / scale > 5e-16
