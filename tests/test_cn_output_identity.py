"""The arithmetic identity behind the column-indexed kernel's MS-family check-node output
(Eqs. 4 and 8), emulated in FP32 with numpy on the CPU.

Edge j of a check receives min(g * min_{i != j} |v_i|, clip) with the sign of the other
edges' parity.  The selection form computes the smallest and second-smallest |v| and picks
per edge.  The kernel instead folds the parity bit into the gain (g > 0), scales every
|v_i| by it, and takes unsigned minima of the resulting bit patterns over the other edges:
the slot pair's partner, a prefix over earlier pair minima and a suffix over later ones,
seeded with the signed clip.  Both rest on two facts pinned here: fl(g x) is monotone in x
for g > 0, and floats of one sign order like their bit patterns as unsigned integers.  The
two forms must give the same bits on every input, including ties, signed zeros, padded
slots (+inf), degree-1 checks, and the smallest gains the library accepts."""
import numpy as np
import pytest

SIGN = np.uint32(0x80000000)
CLIP = np.float32(1e6)


def f2u(x):
    return np.asarray(x, np.float32).view(np.uint32)


def u2f(x):
    return np.asarray(x, np.uint32).view(np.float32)


def selection_form(v, g, par):
    """Smallest / second-smallest |v|, two edges at a time, then a per-edge select; the
    stored value is the negated message, sign = NOT(parity XOR sign(v_j))."""
    a = np.abs(v)
    m1 = m2 = np.float32(np.inf)
    for j in range(0, len(v), 2):
        lo, hi = min(a[j], a[j + 1]), max(a[j], a[j + 1])
        m2 = min(m2, hi, max(m1, lo))
        m1 = min(m1, lo)
    o1 = f2u(min(np.float32(g * m1), CLIP)) | par
    o2 = f2u(min(np.float32(g * m2), CLIP)) | par
    return np.array([(o2 if a[j] == m1 else o1) ^ (~f2u(v[j]) & SIGN) for j in range(len(v))], np.uint32)


def excluded_minimum_form(v, g, par):
    """Sign-carrying scaled magnitudes, unsigned minima over the other edges (pair partner,
    prefix of pair minima, suffix of pair minima seeded with the signed clip)."""
    gs = u2f(f2u(g) | par)
    x = f2u((gs * np.abs(v)).astype(np.float32))
    npr = len(v) // 2
    pm = [min(x[2 * i], x[2 * i + 1]) for i in range(npr)]
    sp = [np.uint32(0)] * npr
    sp[-1] = f2u(CLIP) | par
    for i in range(npr - 2, -1, -1):
        sp[i] = min(sp[i + 1], pm[i + 1])
    out = np.zeros(len(v), np.uint32)
    pre = None
    for i in range(npr):
        o0 = min(x[2 * i + 1], sp[i]) if i == 0 else min(x[2 * i + 1], pre, sp[i])
        o1 = min(x[2 * i], sp[i]) if i == 0 else min(x[2 * i], pre, sp[i])
        pre = pm[0] if i == 0 else min(pre, pm[i])
        out[2 * i] = o0 ^ (~f2u(v[2 * i]) & SIGN)
        out[2 * i + 1] = o1 ^ (~f2u(v[2 * i + 1]) & SIGN)
    return out


GAINS = [1.0, 0.75, 0.3 * 1.1, 2.0 ** -20, float(np.nextafter(np.float32(0), np.float32(1)))]


def _cases(rng, count):
    for _ in range(count):
        dc = int(rng.choice([6, 8, 10]))
        deg = int(rng.integers(1, dc + 1))
        kind = int(rng.integers(0, 4))
        if kind == 0:
            v = rng.normal(0, 3, dc)
        elif kind == 1:   # ties, signed zeros, tiny and clipped-size values
            v = rng.choice([0.0, -0.0, 1.0, -1.0, 2.5, -2.5, 1e-40, -1e-40, 3e6], dc)
        elif kind == 2:   # many exact ties (integer-valued normalised MS messages)
            v = rng.integers(-3, 4, dc) * 0.5
        else:             # wide dynamic range
            v = rng.normal(0, 1, dc) * 10.0 ** rng.integers(-30, 30, dc)
        v = np.asarray(v, np.float32)
        v[deg:] = np.inf                     # padded slots read +inf
        g = np.float32(rng.choice(GAINS + [rng.uniform(2.0 ** -20, 1.0)]))
        par = np.uint32(int(rng.integers(0, 2)) << 31)
        yield v, g, par


@pytest.mark.parametrize("seed", range(4))
def test_excluded_minimum_equals_selection_bitwise(seed):
    rng = np.random.default_rng(seed)
    for v, g, par in _cases(rng, 5000):
        assert np.array_equal(selection_form(v, g, par), excluded_minimum_form(v, g, par)), (v, g, par)


def test_degree_one_check_gets_the_signed_clip():
    v = np.array([2.0, np.inf, np.inf, np.inf, np.inf, np.inf], np.float32)
    for par in (np.uint32(0), SIGN):
        out = excluded_minimum_form(v, np.float32(0.5), par)
        assert out[0] == (f2u(CLIP) | par) ^ (~f2u(v[0]) & SIGN)


def test_a_negative_gain_would_break_the_identity():
    """Why the gain must stay positive (the library requires alpha_min >= 2^-20, so Eq. 7's
    FP32 gain cannot round to zero or below): with a negative gain the scaled values carry
    the wrong sign bit, the clip orders first as an unsigned integer, and the outputs differ
    from the selection form.  (A zero gain has a platform-dependent failure instead: 0 * inf
    on a padded slot is a NaN whose sign bit decides where it orders.)"""
    v = np.array([1.0, 2.0, 3.0, -4.0], np.float32)
    g = np.float32(-0.5)
    assert not np.array_equal(excluded_minimum_form(v, g, np.uint32(0)), selection_form(v, g, np.uint32(0)))


def _worst_base(amin, amaxes):
    """Smallest FP32 base gain a_max - (a_max - a_min) * (float(cnt) * inv_m), inv_m = 1.0f / m,
    over m <= 1024 and 0 <= cnt <= m, both with two roundings and with one (FMA contraction)."""
    from fractions import Fraction
    worst = np.inf
    for m in range(1, 1025):
        inv_m = np.float32(1.0) / np.float32(m)
        frac = (np.arange(m + 1, dtype=np.float32) * inv_m).astype(np.float32)
        for amax in amaxes:
            d = np.float32(amax - amin)
            plain = (amax - (d * frac).astype(np.float32)).astype(np.float32)
            fma = Fraction(float(amax)) - Fraction(float(d)) * Fraction(float(frac.max()))
            worst = min(worst, float(plain.min()), float(fma))
    return worst


AMAXES = np.float32([1.0, np.nextafter(np.float32(1), np.float32(0)), 0.9, 0.5, 2.0 ** -10, 2.0 ** -19])


def test_smallest_accepted_alpha_min_keeps_the_fp32_gain_positive():
    """Eq. 7's base gain as the kernels evaluate it in FP32 stays positive at the library's
    smallest a_min = 2^-20 for every code size m <= 1024 (the library's limit), every
    unsatisfied count and a range of a_max in [a_min, 1] (the automatic ceiling keeps a_max
    there too), whether or not the compiler contracts the product and the difference into one
    FMA.  The bound comes from a worst-case rounding analysis; measured, the gain first
    reaches zero at a_min = 2^-25, so the accepted range keeps a factor-16 margin."""
    amin = np.float32(2.0 ** -20)
    assert _worst_base(amin, list(AMAXES) + [amin]) > 0
    assert _worst_base(np.float32(2.0 ** -24), AMAXES) > 0
    assert _worst_base(np.float32(2.0 ** -25), AMAXES) <= 0
