"""Pins of the oracle's spectral derivatives and single-particle Hamiltonian
against closed forms, brute force and invariants (CPU only)."""
import numpy as np
import pytest

import oracle as O
from paper_1610_07522_gb300 import inputs as IN


def _pw(grid, m, s, twist_free=True):
    """Plane wave e^{i k.r}/sqrt(L^3) in spin component s (built here, by hand)."""
    nx, ny, nz = grid.n
    z, y, x = np.meshgrid(np.arange(nz) * grid.dx[2], np.arange(ny) * grid.dx[1],
                          np.arange(nx) * grid.dx[0], indexing="ij")
    ph = np.exp(2j * np.pi * (m[0] * x / grid.L[0] + m[1] * y / grid.L[1] + m[2] * z / grid.L[2]))
    psi = np.zeros((2, nz, ny, nx), dtype=complex)
    psi[s] = ph / np.sqrt(grid.L[0] * grid.L[1] * grid.L[2])
    return psi


def _kvec(grid, m):
    """Wavenumber of integer mode m, folded to [-n/2, n/2), plus twist."""
    out = []
    for j in range(3):
        mj = ((m[j] + grid.n[j] // 2) % grid.n[j]) - grid.n[j] // 2
        out.append(2 * np.pi * mj / grid.L[j] + grid.theta[j] / grid.L[j])
    return np.array(out)


@pytest.mark.parametrize("n", [4, 5, 6, 8, 12])
def test_derivative_matches_bruteforce_trig_interpolant(n):
    """d_x f by an explicit O(n^2) sum over modes m in [-n/2, n/2) (Nyquist kept)."""
    rng = np.random.default_rng(n)
    grid = O.Grid((n, 3, 2), (0.7, 1.0, 1.0), twist=(0.3, 0.0, 0.0))
    f = rng.standard_normal(grid.shape) + 1j * rng.standard_normal(grid.shape)
    got = O.deriv(f, 0, grid)
    L = grid.L[0]
    xs = np.arange(n) * grid.dx[0]
    ms = [m for m in range(-(n // 2), n - n // 2)]
    want = np.zeros_like(f)
    for a in range(n):
        acc = 0.0
        for m in ms:
            k = 2 * np.pi * m / L
            fh = sum(f[..., b] * np.exp(-1j * k * xs[b]) for b in range(n))
            acc = acc + 1j * (k + grid.theta[0] / L) * fh * np.exp(1j * k * xs[a]) / n
        want[..., a] = acc
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def test_derivative_of_sin_cos_is_exact():
    grid = O.Grid((16, 12, 10), (1.0, 0.5, 2.0))
    z, y, x = np.meshgrid(*(np.arange(grid.n[j]) * grid.dx[j] for j in (2, 1, 0)), indexing="ij")
    kx, ky, kz = 2 * np.pi * 3 / grid.L[0], 2 * np.pi * 2 / grid.L[1], 2 * np.pi / grid.L[2]
    f = np.sin(kx * x) * np.cos(ky * y) * np.cos(kz * z)
    assert np.allclose(O.deriv_real(f, 0, grid), kx * np.cos(kx * x) * np.cos(ky * y) * np.cos(kz * z), atol=1e-12)
    assert np.allclose(O.deriv_real(f, 1, grid), -ky * np.sin(kx * x) * np.sin(ky * y) * np.cos(kz * z), atol=1e-12)
    assert np.allclose(O.deriv_real(f, 2, grid), -kz * np.sin(kx * x) * np.cos(ky * y) * np.sin(kz * z), atol=1e-12)
    assert np.allclose(O.laplacian_real(f, grid), -(kx ** 2 + ky ** 2 + kz ** 2) * f, atol=1e-11)


def test_parseval_and_shift_theorem():
    rng = np.random.default_rng(3)
    grid = O.Grid((8, 6, 5), (1.0, 1.0, 1.0))
    f = rng.standard_normal(grid.shape) + 1j * rng.standard_normal(grid.shape)
    F = O.fft3(f)
    assert abs(np.sum(np.abs(F) ** 2) / grid.G - np.sum(np.abs(f) ** 2)) < 1e-10
    # shift by 2 along x multiplies mode m by e^{-2 pi i m 2 / n}
    Fs = O.fft3(np.roll(f, 2, axis=-1))
    m = np.fft.fftfreq(8, d=1.0 / 8)
    assert np.allclose(Fs, F * np.exp(-2j * np.pi * m * 2 / 8)[None, None, :], atol=1e-11)


@pytest.mark.parametrize("twist", [(0.0, 0.0, 0.0), (0.4, -1.1, 2.5)])
def test_plane_waves_are_exact_eigenfunctions(twist):
    """Uniform U, B and W = 0: h e^{ik.r} chi = (B |k + theta/L|^2 + U) e^{ik.r} chi
    for every k of the grid, the Nyquist modes included."""
    grid = O.Grid((8, 6, 4), (1.0, 1.2, 0.9), twist=twist)
    U = np.full(grid.shape, -37.5)
    B = np.full(grid.shape, 17.25)
    W = np.zeros((3,) + grid.shape)
    modes = [(0, 0, 0), (1, 0, 0), (-4, 0, 0), (4, 3, 2), (-4, -3, -2), (3, -2, 1), (2, 3, -2)]
    for m in modes:
        for s in (0, 1):
            psi = _pw(grid, m, s)
            h = O.apply_h(psi, U, B, W, grid)
            k = _kvec(grid, m)
            e = 17.25 * np.dot(k, k) - 37.5
            assert np.max(np.abs(h - e * psi)) < 1e-12 * max(1.0, abs(e)) * np.max(np.abs(psi))


def test_constant_spin_orbit_field_on_plane_wave():
    """Uniform W: the spin-orbit term on e^{ik.r} chi is ((W x k).sigma) e^{ik.r} chi,
    so h acts as the 2x2 matrix (B k^2 + U) 1 + (W x k).sigma."""
    grid = O.Grid((8, 8, 8), (1.0, 1.0, 1.0), twist=(0.3, 0.2, -0.5))
    Wc = np.array([3.0, -2.0, 1.5])
    U = np.full(grid.shape, -20.0)
    B = np.full(grid.shape, 15.0)
    W = Wc[:, None, None, None] * np.ones((3,) + grid.shape)
    for m in [(1, 0, 0), (0, 2, -1), (-3, 1, 2)]:
        k = _kvec(grid, m)
        c = np.cross(Wc, k)
        Hs = (15.0 * k.dot(k) - 20.0) * np.eye(2) + sum(c[a] * O.SIGMA[a] for a in range(3))
        for chi in (np.array([1.0, 0.0]), np.array([0.3 - 0.2j, 0.8 + 0.1j])):
            psi = chi[0] * _pw(grid, m, 0) + chi[1] * _pw(grid, m, 1)
            h = O.apply_h(psi, U, B, W, grid)
            want = (Hs @ chi)[:, None, None, None] * _pw(grid, m, 0)[0][None]
            assert np.max(np.abs(h - want)) < 1e-11


def _random_fields(grid, rng):
    U = IN.random_smooth_field(grid.n, rng, -40.0, 20.0)
    B = IN.random_smooth_field(grid.n, rng, 20.0, 6.0)
    W = np.stack([IN.random_smooth_field(grid.n, rng, 0.0, 8.0) for _ in range(3)])
    return U, B, W


@pytest.mark.parametrize("twist", [(0.0, 0.0, 0.0), (0.7, -2.0, 1.3)])
def test_h_is_hermitian(twist):
    rng = np.random.default_rng(11)
    grid = O.Grid((8, 6, 10), (1.0, 1.1, 0.8), twist=twist)
    U, B, W = _random_fields(grid, rng)
    a = IN.random_spinors(grid.n, 3, rng)
    b = IN.random_spinors(grid.n, 3, rng)
    ha = O.apply_h(a, U, B, W, grid)
    hb = O.apply_h(b, U, B, W, grid)
    for i in range(3):
        for j in range(3):
            lhs = O.inner(a[i], hb[j], grid)
            rhs = np.conj(O.inner(b[j], ha[i], grid))
            scale = np.sqrt(np.real(O.inner(a[i], a[i], grid)) * np.real(O.inner(hb[j], hb[j], grid)))
            assert abs(lhs - rhs) <= 1e-13 * scale
        assert abs(np.imag(O.inner(a[i], ha[i], grid))) <= 1e-13 * abs(O.inner(a[i], ha[i], grid))


def test_h_drops_no_term():
    """Each of U, B and W changes h psi (guards against a silently dropped field)."""
    rng = np.random.default_rng(5)
    grid = O.Grid((8, 8, 8), (1.0, 1.0, 1.0))
    U, B, W = _random_fields(grid, rng)
    a = IN.random_spinors(grid.n, 1, rng)
    base = O.apply_h(a, U, B, W, grid)
    for U2, B2, W2 in ((U * 1.1, B, W), (U, B * 1.1, W), (U, B, W * 1.1), (U, B, W[[1, 0, 2]])):
        assert np.max(np.abs(O.apply_h(a, U2, B2, W2, grid) - base)) > 1e-3 * np.max(np.abs(base))


def test_translation_invariance():
    rng = np.random.default_rng(9)
    grid = O.Grid((8, 6, 10), (1.0, 1.0, 1.0))
    U, B, W = _random_fields(grid, rng)
    a = IN.random_spinors(grid.n, 2, rng)
    h = O.apply_h(a, U, B, W, grid)
    sh = (2, -1, 3)  # (z, y, x) integer shifts
    roll = lambda f: np.roll(f, sh, axis=(-3, -2, -1))
    hs = O.apply_h(roll(a), roll(U), roll(B), roll(W), grid)
    assert np.max(np.abs(hs - roll(h))) < 1e-12 * np.max(np.abs(h))


def test_dense_h_small_matches_apply():
    rng = np.random.default_rng(2)
    grid = O.Grid((4, 4, 2), (1.0, 1.0, 1.0))
    U, B, W = _random_fields(grid, rng)
    Hd = O.dense_h(U, B, W, grid)
    assert np.max(np.abs(Hd - Hd.conj().T)) < 1e-12 * np.max(np.abs(Hd))
    a = IN.random_spinors(grid.n, 1, rng)[0]
    assert np.allclose(Hd @ a.reshape(-1), O.apply_h(a, U, B, W, grid).reshape(-1), atol=1e-10)
