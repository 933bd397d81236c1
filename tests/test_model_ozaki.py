"""NumPy model of the exact-integer digit split used by the FP64 and FP32
forms' tensor-core contractions (documentation of the algorithm, not parity
evidence: the GPU kernels are compared with the oracle in
tests/test_gpu_split_gemm.py).

Each row of an operand is scaled by 2^E (|x| < 2^E over the row) and x is
written as X = round(|x| 2^(8S - E)) in balanced base-256 digits a_0 in
[0, 256], a_s in [-128, 127] (s >= 1), then given the sign of x (so
|a_0| <= 256, |a_s| <= 128), so that
    x ~ 2^E sum_s a_s 2^-8(s+1),   |error| <= 2^(E - 8S - 1).
Digit products of total weight g = s + t are summed together; per K value
their sum is bounded by 2^16 (g = 0) or (g + 3) 2^14 (g >= 1), so a segment
of 128 K values stays below 2^24 and sums exactly in FP32.  The pins: the
digit ranges and the reconstruction bound (including exact powers of two,
zeros and the round-up carry), the per-weight bound and FP32 exactness of a
worst-case segment, exact products for operands of one or two digits, and
the error of the kept products (weight <= S - 1) on random data."""
import numpy as np
import pytest


def row_exponent(row):
    m = np.max(np.abs(row))
    if m == 0:
        return 0
    _, e = np.frexp(m)          # m = f 2^e, f in [0.5, 1): |x| < 2^e
    return int(e)


def digits(x, E, S):
    """Balanced base-256 digits of |x| 2^(8S - E) rounded, with x's sign."""
    X = int(round(abs(x) * 2.0 ** (8 * S - E)))   # exact: a power-of-two scaling, then rounding
    d = [0] * S
    for s in range(S - 1, 0, -1):
        v = X & 255
        X >>= 8
        if v >= 128:
            v -= 256
            X += 1
        d[s] = v
    d[0] = X
    sgn = -1 if x < 0 else 1
    return [sgn * v for v in d]


def split_rows(A, S):
    E = [row_exponent(r) for r in A]
    D = np.zeros((S,) + A.shape, dtype=np.int64)
    for i, r in enumerate(A):
        for k, x in enumerate(r):
            D[:, i, k] = digits(float(x), E[i], S)
    return D, np.array(E)


def reconstruct(D, E, S):
    w = np.array([2.0 ** (-8 * (s + 1)) for s in range(S)])
    return np.einsum("s,sik->ik", w, D.astype(np.float64)) * np.ldexp(1.0, E)[:, None]


@pytest.mark.parametrize("S", [4, 6])
def test_digit_ranges_and_reconstruction(S):
    rng = np.random.default_rng(1)
    A = rng.standard_normal((6, 200)) * np.exp(rng.uniform(-20, 20, (6, 1)))
    A[0, :5] = [0.0, 1.0, -0.5, 2.0 ** -30, np.nextafter(1.0, 0.0)]
    D, E = split_rows(A, S)
    assert D[0].min() >= -256 and D[0].max() <= 256
    assert D[1:].min() >= -128 and D[1:].max() <= 128
    err = np.abs(reconstruct(D, E, S) - A)
    assert np.all(err <= np.ldexp(1.0, E - 8 * S - 1)[:, None] * (1 + 1e-12))


def test_round_up_carries_into_the_top_digit():
    # just below 2^E: X rounds up to 2^(8S), the top digit becomes 256
    S = 6
    x = np.nextafter(1.0, 0.0)
    d = digits(x, 0, S)
    assert d == [256, 0, 0, 0, 0, 0]


def test_weight_sums_bounded_and_exact_in_fp32():
    """Worst case per weight: every digit at its largest magnitude (256, 128)
    with matching signs; 128 values of K give |G_g| <= 2^24, exact in float32."""
    S = 6
    top, rest = 256, -128
    for g in range(S):
        per_k = sum((top if s == 0 else rest) * (top if g - s == 0 else rest)
                    for s in range(g + 1))
        bound = 2 ** 16 if g == 0 else (g + 3) * 2 ** 14
        assert abs(per_k) <= bound
        seg = 128 * per_k
        assert abs(seg) <= 2 ** 24
        acc = np.float32(0.0)
        for _ in range(128):
            acc = np.float32(acc + np.float32(per_k))
        assert float(acc) == seg


@pytest.mark.parametrize("bits", [8, 15])
def test_one_and_two_digit_integers_multiply_exactly(bits):
    rng = np.random.default_rng(bits)
    km = 2 ** bits - 1
    ka = rng.integers(-km, km + 1, size=(5, 64))
    kb = rng.integers(-km, km + 1, size=(7, 64))
    ka[:, 0] = km
    kb[:, 0] = km
    sc = 2.0 ** -(bits + 1)
    S = 6
    Da, Ea = split_rows(ka * sc, S)
    Db, Eb = split_rows(kb * sc, S)
    G = sum(np.einsum("ik,jk->ij", Da[s], Db[t]) * 2.0 ** (-8 * (s + t))
            for s in range(S) for t in range(S) if s + t <= S - 1)
    got = G * np.ldexp(1.0, Ea[:, None] + Eb[None, :] - 16)
    assert np.array_equal(got, (ka @ kb.T) * sc * sc)


def test_kept_products_error_on_random_data():
    """The weight <= S - 1 products of Gaussian rows of 4096 values agree with
    the FP64 product to 1e-13 (S = 6) and 1e-8 (S = 4) of the largest entry."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((8, 4096))
    B = rng.standard_normal((6, 4096))
    want = A @ B.T
    for S, tol in ((6, 1e-13), (4, 1e-8)):
        Da, Ea = split_rows(A, S)
        Db, Eb = split_rows(B, S)
        G = sum(np.einsum("ik,jk->ij", Da[s], Db[t]).astype(np.float64) * 2.0 ** (-8 * (s + t))
                for s in range(S) for t in range(S) if s + t <= S - 1)
        got = G * np.ldexp(1.0, Ea[:, None] + Eb[None, :] - 16)
        assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))
