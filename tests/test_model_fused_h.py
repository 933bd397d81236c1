"""NumPy models of the arithmetic behind the FP32 forms' fused h psi and
their float-pair reductions (documentation of the algorithms, checked against
the oracle and exact rational arithmetic; the GPU kernels themselves are
compared with the oracle in tests/test_gpu_parity.py):

* the spin-orbit matrices A_j = (sigma x W)_j the kernels apply to a spinor,
  written out per axis, are sum_ik eps_ijk W_i sigma_k, the matrices of the
  oracle's W.(-i)(nabla x sigma) term;
* h psi = U psi + sum_j [ -(i/2) A_j d_j psi + d_j ( -B d_j psi - (i/2) A_j psi ) ]:
  the share of each axis j needs only derivatives along j, so one pass per
  axis (derivative, pointwise terms, derivative of the flux) sums to the
  oracle's h psi;
* a sum of products of floats kept as a float pair (the product exact as
  p + e with e from an FMA, p added by TwoSum, the errors in the low part)
  is within a few 2^-48 of the exact sum.
"""
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1610_07522_gb300 import inputs as IN


def apply_A(j, W, v0, v1):
    """The kernels' A_j (sigma x W)_j on the spinor (v0, v1), as written there."""
    wx, wy, wz = W
    if j == 0:
        return -wy * v0 - 1j * wz * v1, 1j * wz * v0 + wy * v1
    if j == 1:
        return wx * v0 - wz * v1, -wz * v0 - wx * v1
    return (wy + 1j * wx) * v1, (wy - 1j * wx) * v0


def test_spin_orbit_matrices_are_sigma_cross_W():
    rng = np.random.default_rng(3)
    W = rng.standard_normal(3)
    for j in range(3):
        want = sum(O.levi_civita(i, j, k) * W[i] * O.SIGMA[k]
                   for i in range(3) for k in range(3))
        got = np.zeros((2, 2), dtype=complex)
        for c in range(2):
            e = np.zeros(2)
            e[c] = 1.0
            got[:, c] = apply_A(j, W, e[0], e[1])
        assert np.max(np.abs(got - want)) < 1e-15


@pytest.mark.parametrize("shape,twist", [((8, 12, 16), (0.0, 0.0, 0.0)),
                                         ((12, 8, 8), (0.7, -1.9, 2.5))])
def test_per_axis_shares_sum_to_h(shape, twist):
    g = O.Grid(shape, (1.0, 1.0, 1.0), twist)
    rng = np.random.default_rng(5)
    psi = IN.random_spinors(g.n, 2, rng)
    U = IN.random_smooth_field(g.n, rng, -40.0, 30.0)
    B = IN.random_smooth_field(g.n, rng, 20.0, 6.0)
    W = np.stack([IN.random_smooth_field(g.n, rng, 0.0, 10.0) for _ in range(3)])
    want = O.apply_h(psi, U, B, W, g)
    h = U * psi
    for j in range(3):
        G = O.deriv(psi, j, g)
        a0, a1 = apply_A(j, W, G[:, 0], G[:, 1])
        L = np.stack([-0.5j * a0, -0.5j * a1], axis=1)          # -(i/2) A_j d_j psi
        b0, b1 = apply_A(j, W, psi[:, 0], psi[:, 1])
        F = -B * G + np.stack([-0.5j * b0, -0.5j * b1], axis=1)  # -B d_j psi - (i/2) A_j psi
        h = h + L + O.deriv(F, j, g)
    assert np.max(np.abs(h - want)) < 1e-12 * np.max(np.abs(want))


def f32(x):
    return np.float32(x)


def acc_pair(terms):
    """The kernels' float-pair sum of products a b (float32 inputs)."""
    hi, lo = f32(0.0), f32(0.0)
    for a, b in terms:
        p = f32(a * b)
        e = f32(np.float64(a) * np.float64(b) - np.float64(p))   # the FMA's exact error
        s = f32(hi + p)
        bb = f32(s - hi)
        err = f32(f32(hi - f32(s - bb)) + f32(p - bb))
        hi = s
        lo = f32(lo + f32(err + e))
    return Fraction(float(hi)) + Fraction(float(lo))


@pytest.mark.parametrize("seed,cancel", [(1, False), (2, True), (3, True)])
def test_float_pair_sum_of_products(seed, cancel):
    rng = random.Random(seed)
    n = 3000
    terms = []
    for k in range(n):
        a = f32(rng.uniform(-1, 1) * 2.0 ** rng.randint(-6, 6))
        b = f32(rng.uniform(-1, 1) * 2.0 ** rng.randint(-6, 6))
        if cancel and k % 2:             # near-cancelling pairs, as in J and <psi|h psi>
            a, b = terms[-1][0], f32(-terms[-1][1] * (1 + 2.0 ** -20))
        terms.append((a, b))
    exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in terms)
    got = acc_pair(terms)
    mags = sum(abs(Fraction(float(a)) * Fraction(float(b))) for a, b in terms)
    u = Fraction(1, 2 ** 24)
    assert abs(got - exact) <= 4 * u * u * (n + 1) * mags
    # and far better than a float32 sum
    plain = f32(0.0)
    for a, b in terms:
        plain = f32(plain + f32(a * b))
    assert abs(got - exact) < abs(Fraction(float(plain)) - exact) or got == exact
