"""NumPy model of the split-BF16 precision forms (CPU).

The tensor-core forms write each FP32 value x as BF16 pieces
x = x_0 + x_1 (+ x_2), x_0 = bf16(x), x_1 = bf16(x - x_0), x_2 = bf16(x - x_0 - x_1)
(round to nearest even), and form a product sum from the piece products of
total weight at most nsplit - 1: three products for two pieces (x3), six for
three (x6).  This model checks the representation error of the pieces and
the error of such product sums against the exact FP64 sum of the FP32
inputs, with the accumulation in FP64 so that only the splitting is
measured (the tensor cores accumulate in FP32; that part is bounded by
capping the accumulation length, which the GPU tests cover)."""
import numpy as np
import pytest


def bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even), as float32."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def split(x, n):
    x = np.asarray(x, dtype=np.float32)
    pieces, r = [], x
    for _ in range(n):
        p = bf16(r)
        pieces.append(p)
        r = (r - p).astype(np.float32)
    return pieces


PRODUCTS = {2: [(0, 0), (0, 1), (1, 0)],
            3: [(0, 0), (0, 1), (1, 0), (1, 1), (0, 2), (2, 0)]}


def split_dot(a, b, n):
    pa, pb = split(a, n), split(b, n)
    return sum(np.dot(pa[i].astype(np.float64), pb[j].astype(np.float64)) for i, j in PRODUCTS[n])


def test_bf16_rounding_model():
    x = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 1e-20, 6.5e4], dtype=np.float32)
    y = bf16(x)
    # 8 significant bits survive (half an ulp is 2^-8 relative); ties to even
    assert y[0] == 1.0 and y[1] == 1.0 and y[2] == np.float32(1.0078125)
    assert np.all(np.abs(y - x) <= 2.0 ** -8 * np.abs(x))


@pytest.mark.parametrize("n,bound", [(2, 2.0 ** -16), (3, 2.0 ** -24)])
def test_pieces_represent_the_value(n, bound):
    rng = np.random.default_rng(n)
    x = (rng.standard_normal(100000) * 10.0 ** rng.uniform(-6, 6, 100000)).astype(np.float32)
    s = sum(p.astype(np.float64) for p in split(x, n))
    rel = np.abs(s - x.astype(np.float64)) / np.abs(x.astype(np.float64))
    assert np.max(rel) <= bound


@pytest.mark.parametrize("n,bound", [(2, 2.0 ** -14), (3, 2.0 ** -21)])
def test_split_product_sums(n, bound):
    """Sum of piece products vs the exact sum of the FP32 products, relative
    to sum |a_k b_k| (the scale of the rounding of any such sum)."""
    rng = np.random.default_rng(10 + n)
    for K in (16, 4096):
        a = rng.standard_normal((8, K)).astype(np.float32)
        b = rng.standard_normal((8, K)).astype(np.float32)
        for r in range(8):
            exact = np.dot(a[r].astype(np.float64), b[r].astype(np.float64))
            scale = np.dot(np.abs(a[r]).astype(np.float64), np.abs(b[r]).astype(np.float64))
            assert abs(split_dot(a[r], b[r], n) - exact) <= bound * scale


def test_x6_is_much_closer_than_x3():
    rng = np.random.default_rng(3)
    a = rng.standard_normal(2048).astype(np.float32)
    b = rng.standard_normal(2048).astype(np.float32)
    exact = np.dot(a.astype(np.float64), b.astype(np.float64))
    e3 = abs(split_dot(a, b, 2) - exact)
    e6 = abs(split_dot(a, b, 3) - exact)
    assert e6 < e3 / 100
