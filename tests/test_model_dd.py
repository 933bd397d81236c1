"""NumPy / integer models of the bit-level arithmetic behind the FP64 form's
derivative and pointwise kernels (documentation of the algorithms, checked
against exact rational arithmetic; the GPU kernels themselves are compared
with the oracle in tests/test_gpu_parity.py):

* double -> float pair: hi = the double's pattern rounded at bit 29 (half up,
  a carry into the exponent being the correct rounding), lo = the pattern
  difference, an exact integer count of units of the double's last place,
  converted once to float;
* float pair -> double: hi widened exactly, lo counted in units of the last
  place of hi's double, added to hi's pattern (the unit of the binade below
  when |hi| is a power of two and the sum decreases);
* n / d for n < 2^31 by the invariant multiplier m = ceil(2^p / d),
  p = 31 + ceil(log2 d), q = (n m) >> p (Granlund and Montgomery 1994);
* the derivative along one axis as the circulant matrix D[m][q] =
  d[(m - q) mod n], d[r] = (i/n) sum_a kappa_a e^{2 pi i a r / n}, applied as
  the real 2n x 2n operator on interleaved (re, im) storage, equal to the
  oracle's FFT derivative.
"""
import math
import random
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle as O


def f32(x):
    return struct.unpack("<f", struct.pack("<f", x))[0]


def bits64(x):
    return struct.unpack("<q", struct.pack("<d", x))[0]


def from64(b):
    return struct.unpack("<d", struct.pack("<q", b))[0]


def bits32(x):
    return struct.unpack("<I", struct.pack("<f", x))[0]


def from32(b):
    return struct.unpack("<f", struct.pack("<I", b & 0xFFFFFFFF))[0]


def split(x):
    """double -> (hi, lo) floats as the kernels do it in the normal range."""
    P = bits64(x)
    e = (P >> 52) & 0x7FF
    assert 949 <= e <= 1149
    Ph = (P + (1 << 28)) & ~((1 << 29) - 1)
    sgn = -1.0 if P < 0 else 1.0
    hi = from64(Ph)                     # exactly a float
    assert f32(hi) == hi
    dl = (P & 0x7FFFFFFFFFFFFFFF) - (Ph & 0x7FFFFFFFFFFFFFFF)
    lo = sgn * f32(float(dl)) * 2.0 ** (e - 1075)   # one rounding (int -> float)
    return f32(hi), f32(lo)


def join(hi, lo):
    """(hi, lo) -> double as the kernels do it for normalised pairs."""
    uh, ul = bits32(hi), bits32(lo)
    mh, ml = uh & 0x7FFFFFFF, ul & 0x7FFFFFFF
    eh, el = mh >> 23, ml >> 23
    neg = uh >> 31
    if ml == 0:
        hd = (mh << 29) + (896 << 52)
    else:
        assert 1 <= eh <= 254 and 1 <= el <= 254 and eh - el >= 24
        hd = (mh << 29) + (896 << 52)
        sig = (ul & 0x7FFFFF) | 0x800000
        same = ((uh ^ ul) >> 31) == 0
        down = (not same) and (mh & 0x7FFFFF) == 0
        sh = 29 - (eh - el) + (1 if down else 0)
        if sh >= 0:
            K = sig << sh
        else:
            r = -sh
            K = 0 if r > 25 else ((sig >> (r - 1)) + 1) >> 1
        hd = hd + K if same else hd - K
    v = from64(hd)
    return -v if neg else v


def two_sum_f(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def normalised(h, l):
    """The pair fast_two_sum returns: hi = fl(h + l), lo the exact rest."""
    return two_sum_f(f32(h), f32(l))


def ulp(x):
    """Last place of a double."""
    return math.ulp(x)


def fulp(h):
    """Last place of a (normal) float."""
    return 2.0 ** (math.frexp(h)[1] - 24)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_split_is_exact_to_the_float_rounding_of_the_rest(seed):
    rng = random.Random(seed)
    for _ in range(4000):
        # the integer route's range, 2^-74 <= |x| < 2^127 (outside it the
        # kernels convert through FP64)
        x = rng.choice([-1.0, 1.0]) * rng.uniform(0.5, 1.0) * 2.0 ** rng.randint(-73, 127)
        hi, lo = split(x)
        assert abs(lo) <= fulp(hi) / 2          # hi is x rounded to 24 bits
        rest = Fraction(x) - Fraction(hi)       # exact
        assert abs(Fraction(lo) - rest) <= Fraction(fulp(lo)) / 2   # lo = fl(rest)
        assert abs(Fraction(hi) + Fraction(lo) - Fraction(x)) <= Fraction(abs(x)) * Fraction(1, 2 ** 47)


def test_split_rounds_up_across_a_binade():
    x = from64(bits64(2.0) - 1)        # just below 2: the top 24 bits round up to 2
    hi, lo = split(x)
    assert hi == 2.0 and lo < 0 and hi + lo == x


def _edge_pairs(rng):
    out = []
    for _ in range(3000):
        e = rng.randint(-60, 60)
        h = rng.uniform(1, 2) * 2.0 ** e * rng.choice([-1, 1])
        l = rng.uniform(-0.5, 0.5) * fulp(f32(h)) * rng.choice([1, 2.0 ** -rng.randint(0, 30)])
        out.append(normalised(h, l))
    for e in (-40, -1, 0, 1, 17, 60):          # hi a power of two, lo of either sign
        for frac in (0.5, 0.25, 2.0 ** -13, 2.0 ** -30, 0.4999999):
            for s in (1.0, -1.0):
                h = 2.0 ** e
                out.append(normalised(h, s * frac * fulp(h)))
                out.append(normalised(-h, s * frac * fulp(h)))
    return out


@pytest.mark.parametrize("seed", [4, 5])
def test_join_is_the_rounded_sum(seed):
    rng = random.Random(seed)
    for hi, lo in _edge_pairs(rng):
        got = join(hi, lo)
        exact = Fraction(hi) + Fraction(lo)
        # within half a unit of the double's last place of the result (ties either way)
        assert abs(Fraction(got) - exact) <= Fraction(ulp(got)) / 2, (hi, lo, got)


def test_join_below_a_power_of_two_uses_the_finer_unit():
    h = 1.0
    lo = -f32(2.0 ** -30 + 2.0 ** -52)   # the sum lies in [0.5, 1): unit 2^-53
    hi, lo = normalised(h, lo)
    assert hi == 1.0 and lo < 0
    got = join(hi, lo)
    assert Fraction(got) == Fraction(hi) + Fraction(lo)   # representable: exact


@pytest.mark.parametrize("d", [2, 3, 7, 8, 12, 20, 24, 31, 32, 48, 64, 576, 1000, 65535, 2 ** 31 - 1])
def test_invariant_divisor(d):
    L = (d - 1).bit_length()
    p = 31 + L
    m = -(-(1 << p) // d)
    assert m < 2 ** 32
    rng = random.Random(d)
    for n in [0, 1, d - 1, d, d + 1, 2 ** 31 - 1] + [rng.randrange(2 ** 31) for _ in range(2000)]:
        assert ((n * m) >> 32) >> (p - 32) == n // d


def circulant_operator(n, L, theta):
    a = np.arange(n)
    mm = np.where(a < (n + 1) // 2, a, a - n)
    kap = (2 * np.pi * mm + theta) / L
    r = np.arange(n)
    d = 1j / n * np.exp(2j * np.pi * np.outer(r, a) / n) @ kap
    D = d[(np.arange(n)[:, None] - np.arange(n)[None, :]) % n]
    R = np.zeros((2 * n, 2 * n))
    R[0::2, 0::2] = D.real
    R[0::2, 1::2] = -D.imag
    R[1::2, 0::2] = D.imag
    R[1::2, 1::2] = D.real
    return D, R


@pytest.mark.parametrize("shape,dx,twist", [((8, 12, 16), (1.0, 0.8, 1.2), (0.0, 0.0, 0.0)),
                                            ((24, 20, 8), (1.0, 1.0, 0.9), (0.7, -1.3, 2.2))])
def test_circulant_operator_is_the_fft_derivative(shape, dx, twist):
    g = O.Grid(shape, dx, twist)
    rng = np.random.default_rng(11)
    nz, ny, nx = g.shape
    f = rng.standard_normal((nz, ny, nx)) + 1j * rng.standard_normal((nz, ny, nx))
    for j in range(3):
        n = g.n[j]
        D, R = circulant_operator(n, g.L[j], g.theta[j])
        want = O.deriv(f, j, g)
        ax = 2 - j                                  # numpy axis of spatial axis j
        got = np.moveaxis(np.tensordot(D, np.moveaxis(f, ax, 0), axes=(1, 0)), 0, ax)
        assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))
        # the real operator on interleaved storage is the same map
        line = np.moveaxis(f, ax, -1).reshape(-1, n)
        inter = np.stack([line.real, line.imag], axis=-1).reshape(-1, 2 * n)
        out = inter @ R.T
        outc = (out[:, 0::2] + 1j * out[:, 1::2]).reshape(np.moveaxis(f, ax, -1).shape)
        assert np.max(np.abs(np.moveaxis(outc, -1, ax) - want)) < 1e-12 * np.max(np.abs(want))


def dft_operator(n, inverse):
    """The unnormalised DFT of a line as the operator matrix the kernels use:
    D[m][q] = e^{-+2 pi i (m q mod n) / n} (not circulant: it depends on m q)."""
    mq = np.outer(np.arange(n), np.arange(n)) % n
    return np.exp((2j if inverse else -2j) * np.pi * mq / n)


@pytest.mark.parametrize("n", [8, 12, 20, 24, 32])
def test_dft_operators_are_the_fft(n):
    rng = np.random.default_rng(n)
    f = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.allclose(dft_operator(n, False) @ f, np.fft.fft(f), rtol=0, atol=1e-12 * n)
    assert np.allclose(dft_operator(n, True) @ f, n * np.fft.ifft(f), rtol=0, atol=1e-12 * n)
    # the derivative's circulant form is F^-1 diag(i kappa) F
    D, _ = circulant_operator(n, 7.0, 0.4)
    a = np.arange(n)
    kap = (2 * np.pi * np.where(a < (n + 1) // 2, a, a - n) + 0.4) / 7.0
    want = dft_operator(n, True) @ np.diag(1j * kap) @ dft_operator(n, False) / n
    assert np.max(np.abs(D - want)) < 1e-12 * np.max(np.abs(want))
