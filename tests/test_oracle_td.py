"""Pins of the time-dependent oracle (oracle/td_oracle.py) against what the
mathematics fixes: eigenvectors of h evolve by the scalar Taylor polynomial
of exp(-i eps dt / hbar c) (plane waves with constant fields, eigenvalue
B |k + theta/L|^2 + U; with a constant W the 2x2 matrix of the spin-orbit
closed form), the series approaches the matrix exponential of the dense h
within the Taylor remainder, the evolution is unitary and reversible to the
truncation order, and the self-consistent evolution conserves the energy of
the functional to second order in dt (the midpoint mean field)."""
import math

import numpy as np
import pytest
from scipy.linalg import expm

import oracle as O
from oracle import td_oracle as T
from paper_1610_07522_gb300 import inputs as IN

P = dict(IN.SLY4)


def _plane_wave(grid, m, spin):
    L = np.array(grid.L)
    k = 2 * np.pi * np.array(m) / L + np.array(grid.theta) / L
    nz, ny, nx = grid.shape
    z, y, x = np.meshgrid(np.arange(nz) * grid.dx[2], np.arange(ny) * grid.dx[1],
                          np.arange(nx) * grid.dx[0], indexing="ij")
    ph = np.exp(1j * (k[0] * x + k[1] * y + k[2] * z))   # periodic part times the twist
    psi = np.zeros((1, 2, nz, ny, nx), dtype=np.complex128)
    psi[0, spin] = ph * np.exp(-1j * (grid.theta[0] / L[0] * x + grid.theta[1] / L[1] * y
                                      + grid.theta[2] / L[2] * z))
    return psi, k


@pytest.mark.parametrize("m,twist", [((1, 0, 0), (0, 0, 0)), ((2, -1, 3), (0.4, -0.7, 1.1)),
                                     ((-4, 4, 0), (0, 0, 0))])
def test_plane_wave_phase(m, twist):
    g = O.Grid((8, 8, 8), (1.0, 1.0, 1.0), twist)
    psi, k = _plane_wave(g, m, 0)
    U0, B0 = -37.5, 18.0
    U = np.full(g.shape, U0)
    B = np.full(g.shape, B0)
    W = np.zeros((3,) + g.shape)
    eps = B0 * float(k @ k) + U0
    for dt in (0.05, 0.2):
        got = T.taylor_step(psi, U, B, W, g, dt)
        want = T.scalar_taylor(-1j * eps * dt / T.HBARC) * psi
        assert np.max(np.abs(got - want)) < 1e-13
        # and the series is the exponential to its remainder |z|^7 / 7!
        z = eps * dt / T.HBARC
        assert (abs(T.scalar_taylor(-1j * z) - np.exp(-1j * z))
                <= abs(z) ** 7 / math.factorial(7) * (1 + 1e-6) + 1e-15)


def test_constant_spin_orbit_two_by_two():
    """Constant W on a plane wave: h acts as (B k^2 + U) + (W x k).sigma on the
    spinor (the spin-orbit closed form), so the propagator is the Taylor
    polynomial of that 2x2 matrix."""
    g = O.Grid((8, 8, 8), (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    psi_up, k = _plane_wave(g, (1, 2, -1), 0)
    psi = psi_up.copy()
    psi[0, 1] = (0.6 - 0.8j) * psi_up[0, 0]
    U0, B0, Wc = -20.0, 21.0, np.array([3.0, -1.5, 2.0])
    U, B = np.full(g.shape, U0), np.full(g.shape, B0)
    W = Wc[:, None, None, None] * np.ones((3,) + g.shape)
    h2 = (B0 * float(k @ k) + U0) * np.eye(2) + np.einsum("i,ijk->jk", np.cross(Wc, k), O.SIGMA)
    dt = 0.15
    z = -1j * dt / T.HBARC
    P2 = sum(np.linalg.matrix_power(z * h2, n) / math.factorial(n) for n in range(7))
    chi = np.array([1.0, 0.6 - 0.8j])
    want = np.einsum("ab,b->a", P2, chi)[None, :, None, None, None] * psi_up[0, 0][None, None]
    got = T.taylor_step(psi, U, B, W, g, dt)
    assert np.max(np.abs(got - want)) < 1e-12


def test_series_approaches_the_dense_exponential():
    rng = np.random.default_rng(3)
    g = O.Grid((4, 4, 4), (1.0, 1.0, 1.0), (0.2, 0.0, -0.3))
    U = IN.random_smooth_field(g.n, rng, -30.0, 10.0)
    B = IN.random_smooth_field(g.n, rng, 20.0, 3.0)
    W = np.stack([IN.random_smooth_field(g.n, rng, 0.0, 4.0) for _ in range(3)])
    H = O.dense_h(U, B, W, g)
    psi = IN.random_spinors(g.n, 2, rng)
    dt = 0.1
    x = np.linalg.norm(H, 2) * dt / T.HBARC
    Uex = expm(-1j * H * dt / T.HBARC)
    got = T.taylor_step(psi, U, B, W, g, dt)
    for a in range(2):
        want = (Uex @ psi[a].reshape(-1)).reshape(psi[a].shape)
        bound = x ** 7 / math.factorial(7) * np.linalg.norm(psi[a]) * 1.01 + 1e-13
        assert np.linalg.norm(got[a] - want) <= bound


def test_unitary_and_reversible_with_a_frozen_field():
    rng = np.random.default_rng(4)
    g = O.Grid((8, 8, 8), (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    U = IN.random_smooth_field(g.n, rng, -40.0, 20.0)
    B = IN.random_smooth_field(g.n, rng, 20.0, 4.0)
    W = np.stack([IN.random_smooth_field(g.n, rng, 0.0, 6.0) for _ in range(3)])
    psi = O.orthonormalize(IN.random_superpositions(g.n, g.dx, 6, rng), g)
    cur = psi
    for _ in range(10):
        cur = T.taylor_step(cur, U, B, W, g, 0.1)
    S = O.overlap(cur, cur, g)
    assert np.max(np.abs(S - np.eye(6))) < 1e-9
    back = cur
    for _ in range(10):
        back = T.taylor_step(back, U, B, W, g, -0.1)
    assert np.max(np.abs(back - psi)) < 1e-9 * np.max(np.abs(psi))


def _start(grid, N, Z, seed):
    w = IN.Workload(name="td", grid=grid, dx=(1.0, 1.0, 1.0), N=N, Z=Z, coulomb=True,
                    twist=(0.3, -0.2, 0.5), seed=seed)
    inp = IN.make_inputs(w)
    g = O.Grid(w.grid, w.dx, w.twist)
    return g, O.initial_state(inp["psi0"], g, P, True)


def _drift(dt, steps):
    g, st = _start((8, 8, 8), 4, 3, 11)
    E0 = O.energy(*[np.stack([O.densities(st.psi[q], g)[i] for q in range(2)]) for i in (0, 1, 3)],
                  P, g, True)["total"]
    # the mean field of the start is that of the states (no damped iteration)
    st.U, st.B, st.W = T.field_of(st.psi, g, P, True)[:3]
    E = E0
    for _ in range(steps):
        E = T.td_step(st, g, P, True, dt)["E"]
    S = [O.overlap(st.psi[q], st.psi[q], g) for q in range(2)]
    return E - E0, S, E0


def test_energy_conserved_to_second_order_and_states_stay_orthonormal():
    d1, S1, E0 = _drift(0.2, 5)
    d2, S2, _ = _drift(0.1, 10)
    assert abs(d1) < 1e-4 * abs(E0)
    ratio = abs(d1) / abs(d2)
    assert 3.0 < ratio < 5.5, ratio                  # second order: halving dt quarters the drift
    for S in S1 + S2:
        assert np.max(np.abs(S - np.eye(S.shape[0]))) < 1e-8
