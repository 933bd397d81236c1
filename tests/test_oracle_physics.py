"""Pins of the oracle's densities, functional, mean fields, Coulomb term and
damped step against closed forms, invariants, published nuclear-matter
properties and finite differences of the energy (CPU only)."""
import numpy as np
import pytest

import oracle as O
from paper_1610_07522_gb300 import inputs as IN

P = dict(IN.SLY4)


def _grid_xyz(grid):
    return np.meshgrid(*(np.arange(grid.n[j]) * grid.dx[j] for j in (2, 1, 0)), indexing="ij")


def _orthonormal_random(grid, I, rng):
    raw = IN.random_superpositions(grid.n, grid.dx, I, rng)
    return O.orthonormalize(raw, grid)


# ----------------------------------------------------------------- densities

def test_density_integrates_to_particle_number():
    rng = np.random.default_rng(1)
    grid = O.Grid((8, 8, 6), (1.0, 1.0, 1.2))
    psi = _orthonormal_random(grid, 5, rng)
    rho, tau, J, divJ = O.densities(psi, grid)
    assert abs(grid.dV * rho.sum() - 5.0) < 1e-12
    assert abs(grid.dV * divJ.sum()) < 1e-10   # a divergence integrates to zero


def test_densities_invariant_under_unitary_mixing_and_phases():
    rng = np.random.default_rng(2)
    grid = O.Grid((8, 6, 8), (1.0, 1.0, 1.0), twist=(0.5, -0.3, 0.9))
    psi = _orthonormal_random(grid, 4, rng)
    X = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    Q, _ = np.linalg.qr(X)
    mixed = np.tensordot(Q, psi, axes=(1, 0)) * np.exp(1j * rng.uniform(0, 6, 4))[:, None, None, None, None]
    a, b = O.densities(psi, grid), O.densities(mixed, grid)
    for x, y in zip(a, b):
        assert np.max(np.abs(x - y)) < 1e-13 * max(1.0, np.max(np.abs(x))) * 10


def test_plane_wave_densities_closed_form():
    """Single plane wave e^{ik.r} chi_up/sqrt(V): rho = 1/V, tau = |k|^2/V,
    J = (k x z_hat)/V (from J_i = Re sum eps_ijk (-i) psi^+ sigma_k d_j psi with
    psi^+ sigma_z psi = |psi|^2).  A spin-saturated pair has J = 0."""
    grid = O.Grid((8, 8, 8), (1.0, 1.0, 1.0), twist=(0.3, -0.6, 0.2))
    labels = [(2, -1, 1, 0)]
    psi = IN.plane_wave_states(grid.n, grid.dx, labels)
    vol = grid.L[0] * grid.L[1] * grid.L[2]
    k = np.array([2 * np.pi * 2 / 8 + 0.3 / 8, -2 * np.pi / 8 - 0.6 / 8, 2 * np.pi / 8 + 0.2 / 8])
    rho, tau, J, divJ = O.densities(psi, grid)
    assert np.allclose(rho, 1 / vol, atol=1e-15)
    assert np.allclose(tau, k.dot(k) / vol, atol=1e-14)
    want = np.cross(k, [0, 0, 1]) / vol
    for i in range(3):
        assert np.allclose(J[i], want[i], atol=1e-15)
    pair = IN.plane_wave_states(grid.n, grid.dx, [(2, -1, 1, 0), (2, -1, 1, 1)])
    _, _, J2, divJ2 = O.densities(pair, grid)
    assert np.max(np.abs(J2)) < 1e-15 and np.max(np.abs(divJ2)) < 1e-14


def test_divJ_closed_form_modulated_wave():
    """psi = (1 + a cos(q y)) e^{i k x} chi_up: J = -k rho y_hat,
    div J = 2 a q k sin(q y)(1 + a cos(q y))."""
    grid = O.Grid((8, 12, 6), (1.0, 1.0, 1.0))
    z, y, x = _grid_xyz(grid)
    k = 2 * np.pi * 1 / grid.L[0]
    q = 2 * np.pi * 2 / grid.L[1]
    a = 0.3
    f = (1 + a * np.cos(q * y)) * np.exp(1j * k * x)
    psi = np.zeros((1, 2) + grid.shape, dtype=complex)
    psi[0, 0] = f
    rho, tau, J, divJ = O.densities(psi, grid)
    assert np.allclose(J[1], -k * np.abs(f) ** 2, atol=1e-13)
    assert np.allclose(J[0], 0, atol=1e-13) and np.allclose(J[2], 0, atol=1e-13)
    assert np.allclose(divJ, 2 * a * q * k * np.sin(q * y) * (1 + a * np.cos(q * y)), atol=1e-12)


# ----------------------------------------------------------------- functional

def _matter(rho_n, rho_p):
    """Energy per nucleon of uniform continuum matter from the oracle's
    energy functional: one cell with the Fermi-gas kinetic densities."""
    grid = O.Grid((1, 1, 1), (1.0, 1.0, 1.0))
    rho = np.array([rho_n, rho_p]).reshape(2, 1, 1, 1)
    tau = 0.6 * (3 * np.pi ** 2 * rho) ** (2 / 3) * rho
    E = O.energy(rho, tau, np.zeros_like(rho), P, grid, coulomb=False)
    return E["total"] / (rho_n + rho_p)


def test_sly4_symmetric_matter_saturation():
    """Published SLy4 nuclear-matter properties (Chabanat et al. 1998):
    saturation density 0.160 fm^-3, E/A = -15.97 MeV, incompressibility 230 MeV,
    m*/m = 0.69 and symmetry energy 32.0 MeV.  Pins every isoscalar coupling
    and the isovector ones through the symmetry energy."""
    rs = np.linspace(0.12, 0.20, 8001)
    e = np.array([_matter(r / 2, r / 2) for r in rs])
    i = int(np.argmin(e))
    r0 = rs[i]
    assert abs(r0 - 0.1595) < 0.0015
    assert abs(e[i] - (-15.97)) < 0.03
    h = 1e-3
    d2 = (_matter((r0 + h) / 2, (r0 + h) / 2) - 2 * e[i] + _matter((r0 - h) / 2, (r0 - h) / 2)) / h ** 2
    K = 9 * r0 ** 2 * d2
    assert abs(K - 229.9) < 2.0
    C = O.coefficients(P)
    mstar = 1.0 / (1.0 + C["tau"][0] * r0 / P["hb2m_n"])
    assert abs(mstar - 0.695) < 0.01
    d = 1e-3
    esym = (_matter(r0 * (1 + d) / 2, r0 * (1 - d) / 2) - e[i]) / d ** 2
    assert abs(esym - 32.0) < 0.3


def test_pure_neutron_matter_is_unbound():
    for r in (0.02, 0.08, 0.16):
        assert _matter(r, 0.0) > 0.0


def test_gradient_terms_closed_form():
    """rho_n = rho_p = rbar + a cos(2 pi x / L):  int rho_0 Delta rho_0 = -(2 pi/L)^2 (2a)^2 V/2,
    and the isovector part vanishes."""
    grid = O.Grid((12, 4, 4), (1.0, 1.0, 1.0))
    z, y, x = _grid_xyz(grid)
    q = 2 * np.pi / grid.L[0]
    r = 0.04 + 0.01 * np.cos(q * x)
    rho = np.stack([r, r])
    tau = np.zeros_like(rho)
    E = O.energy(rho, tau, np.zeros_like(rho), P, grid, coulomb=False)
    C = O.coefficients(P)
    vol = grid.L[0] * grid.L[1] * grid.L[2]
    want = C["drho"][0] * (-(q ** 2) * (2 * 0.01) ** 2 * vol / 2)
    assert abs(E["drho"] - want) < 1e-12 * abs(want)


def test_spin_orbit_energy_closed_form():
    """Neutron state (1 + a cos(q y)) e^{ikx} chi_up, no protons:
    E_nJ = (C_0 + C_1) int rho div J with the closed-form rho and div J."""
    grid = O.Grid((8, 12, 4), (1.0, 1.0, 1.0))
    z, y, x = _grid_xyz(grid)
    k = 2 * np.pi / grid.L[0]
    q = 2 * np.pi / grid.L[1]
    a = 0.4
    f = (1 + a * np.cos(q * y)) * np.exp(1j * k * x) * 0.1
    psi = np.zeros((1, 2) + grid.shape, dtype=complex)
    psi[0, 0] = f
    rho_n, tau_n, J, divJ_n = O.densities(psi, grid)
    rho = np.stack([rho_n, np.zeros_like(rho_n)])
    tau = np.stack([tau_n, np.zeros_like(rho_n)])
    divJ = np.stack([divJ_n, np.zeros_like(rho_n)])
    E = O.energy(rho, tau, divJ, P, grid, coulomb=False)
    C = O.coefficients(P)
    rc = 0.01 * (1 + a * np.cos(q * y)) ** 2
    dc = 0.01 * 2 * a * q * k * np.sin(q * y) * (1 + a * np.cos(q * y))
    want = (C["nJ"][0] + C["nJ"][1]) * grid.dV * np.sum(rc * dc)
    assert abs(E["nJ"] - want) < 1e-12 * max(abs(want), 1e-6) + 1e-14


def test_coulomb_single_mode_closed_form():
    """rho_p = rbar + a cos(2 pi x/L): V_C = 4 pi e^2 a/(2 pi/L)^2 cos(2 pi x/L);
    E_C = 1/2 int rho_p V_C = pi e^2 a^2 V / q^2."""
    grid = O.Grid((16, 4, 4), (1.0, 1.0, 1.0))
    z, y, x = _grid_xyz(grid)
    q = 2 * np.pi / grid.L[0]
    a = 0.005
    rp = 0.02 + a * np.cos(q * x)
    V = O.coulomb_potential(rp, grid, P["e2"])
    assert np.allclose(V, 4 * np.pi * P["e2"] * a / q ** 2 * np.cos(q * x), atol=1e-13)
    rho = np.stack([np.zeros_like(rp), rp])
    E = O.energy(rho, np.zeros_like(rho), np.zeros_like(rho), P, grid, coulomb=True)
    vol = grid.L[0] * grid.L[1] * grid.L[2]
    want = 0.5 * 4 * np.pi * P["e2"] * a ** 2 / q ** 2 * vol / 2
    assert abs(E["coul"] - want) < 1e-12 * want


@pytest.mark.parametrize("coulomb", [False, True])
def test_mean_fields_are_the_energy_gradient(coulomb):
    """dE/d eta along psi + eta dpsi equals sum_q sum_alpha 2 Re <dpsi|h_q psi>
    with h built from the oracle's U, B, W: ties every mean-field term
    (including Coulomb and the density dependence) to the energy functional."""
    rng = np.random.default_rng(7)
    grid = O.Grid((8, 8, 8), (1.0, 1.0, 1.0), twist=(0.2, -0.4, 0.1))
    psi = [0.9 * IN.random_superpositions(grid.n, grid.dx, I, rng) / 8 for I in (3, 2)]
    dpsi = [IN.random_superpositions(grid.n, grid.dx, I, rng) / 8 for I in (3, 2)]

    def E_of(ps):
        d = [O.densities(ps[q], grid) for q in range(2)]
        rho = np.stack([d[q][0] for q in range(2)])
        tau = np.stack([d[q][1] for q in range(2)])
        divJ = np.stack([d[q][3] for q in range(2)])
        return O.energy(rho, tau, divJ, P, grid, coulomb)["total"], (rho, tau, divJ)

    E0, (rho, tau, divJ) = E_of(psi)
    U, B, W = O.mean_fields(rho, tau, divJ, P, grid, coulomb)
    grad = 0.0
    for q in range(2):
        h = O.apply_h(psi[q], U[q], B[q], W[q], grid)
        grad += 2 * np.real(np.sum(O.inner(dpsi[q], h, grid)))
    eta = 1e-4
    Ep, _ = E_of([psi[q] + eta * dpsi[q] for q in range(2)])
    Em, _ = E_of([psi[q] - eta * dpsi[q] for q in range(2)])
    fd = (Ep - Em) / (2 * eta)
    assert abs(fd - grad) < 1e-6 * abs(grad)


# ----------------------------------------------------------------- damped step

def test_damped_step_closed_form_on_plane_wave_mixture():
    """Uniform U, B (B != hb2m), W = 0, psi = c1 pw(k1) up + c2 pw(k2) down:
    eps = sum |c|^2 e, phi = psi - x0 sum_i (e_i - eps) c_i pw_i / (E0 + hb2m |k_i|^2),
    and <h^2> - <h>^2 = sum |c|^2 e^2 - eps^2."""
    grid = O.Grid((8, 8, 8), (1.0, 1.0, 1.0), twist=(0.4, 0.0, -0.7))
    labels = [(1, 0, 2, 0), (-2, 3, 0, 1)]
    pw = IN.plane_wave_states(grid.n, grid.dx, labels)
    c = np.array([0.6 + 0.2j, -0.3 + 0.7j]); c = c / np.linalg.norm(c)
    psi = (c[0] * pw[0] + c[1] * pw[1])[None]
    U = np.full(grid.shape, -30.0); B = np.full(grid.shape, 14.0)
    W = np.zeros((3,) + grid.shape)
    ks = [np.array([2 * np.pi * 1 / 8 + 0.4 / 8, 0.0, 2 * np.pi * 2 / 8 - 0.7 / 8]),
          np.array([-2 * np.pi * 2 / 8 + 0.4 / 8, 2 * np.pi * 3 / 8, -0.7 / 8])]
    e = np.array([14.0 * k.dot(k) - 30.0 for k in ks])
    hpsi = O.apply_h(psi, U, B, W, grid)
    eps, hn2 = O.sp_energies(psi, hpsi, grid)
    eps_want = np.sum(np.abs(c) ** 2 * e)
    assert abs(eps[0] - eps_want) < 1e-12 * abs(eps_want)
    assert abs(hn2[0] - eps[0] ** 2 - (np.sum(np.abs(c) ** 2 * e ** 2) - eps_want ** 2)) < 1e-9
    hb2m, x0, E0 = 20.73553, 0.45, 100.0
    phi = O.damped_step(psi, hpsi, eps, grid, hb2m, x0, E0)
    want = psi[0] - x0 * sum((e[i] - eps_want) * c[i] * pw[i] / (E0 + hb2m * ks[i].dot(ks[i])) for i in range(2))
    assert np.max(np.abs(phi[0] - want)) < 1e-13
    assert abs(O.convergence_measure([eps], [hn2]) - np.sqrt(np.sum(np.abs(c) ** 2 * e ** 2) - eps_want ** 2)) < 1e-7
