"""Plain FP64 CPU oracle of the damped-gradient Skyrme-DFT iteration
(Afibuzzaman, Schuetrumpf, Aktulga, "Scalable Nuclear Density Functional
Theory with Sky3D", arXiv 1610.07522).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or call this module.  It shares
no code with the CUDA path (it imports nothing from the product package) and
is written for a reader checking it against the paper, not for speed: every
derivative is the 3D-FFT definition, every matrix is formed in full.

What the paper fixes and where (section / equation):
  * one-body equation h_q psi = eps psi ............ Sec. 2.1, Eq. Schroedinger
  * convergence measure (mean energy variance) ..... Sec. 2.1, Eq. convergence
  * Skyrme functional (schematic) .................. Sec. 2.1, Eq. Skyrme
  * densities rho, J, tau .......................... Sec. 2.1, Eqs. rho, curr, tau
  * damped gradient step ........................... Sec. 2.2, Eq. dampstep
  * derivatives and Coulomb by FFT ................. Sec. 2.2 (text after Eq. dampstep)
  * flow of one iteration (steps 2-5) .............. Sec. 2.2, Fig. 1
  * overlap and Hamiltonian matrices ............... Sec. 3.3.1, Eqs. normmatrix, hammatrix
  * lower triangle only ............................ Sec. 3.3.1, Fig. 3
  * Loewdin orthonormalisation C = I^{-1/2} ........ Sec. 3.3.2, Eqs. Loewedin, orthmatvec
  * recombination psi = (C Z) phi .................. Sec. 3.3.3, Fig. 3

Readings where the paper is schematic or silent (each also listed in the
design notes): standard isoscalar/isovector form of the Skyrme functional
with the usual (t, x, W0) coefficients; symmetrised spin-orbit operator;
Nyquist wavenumber kept in every spinor derivative; real part taken for
derivatives of real fields; rho_0^alpha terms set to 0 where rho_0 < 1e-30;
J taken as the real part of its defining expression; step operator taken
literally as delta/(T + E0); exact Rayleigh-Ritz (Loewdin C from the overlap
of phi, then Z from C^H H C) instead of the paper's combined C^T Z^H with Z
from the non-orthonormal H (which the paper notes differs only during the
iteration, Sec. 3.3.3); Coulomb without exchange, zero mode removed
(uniform neutralising background).

Array layouts: spinors [I, 2, nz, ny, nx] complex128, x fastest (Sec. 3.1
``psi(V, A)``); fields [nz, ny, nx] float64; vector fields [3, nz, ny, nx]
with components (x, y, z).
"""
from __future__ import annotations

import numpy as np

AXES3 = (-3, -2, -1)

# Pauli matrices sigma_x, sigma_y, sigma_z (standard representation).
SIGMA = np.array([[[0, 1], [1, 0]],
                  [[0, -1j], [1j, 0]],
                  [[1, 0], [0, -1]]], dtype=np.complex128)


def levi_civita(i, j, k):
    """epsilon_ijk for i, j, k in {0, 1, 2}."""
    return (i - j) * (j - k) * (k - i) // 2


# --------------------------------------------------------------------------
# Grid and spectral derivatives (Sec. 2.2: equidistant periodic grid,
# derivatives "using FFTs")
# --------------------------------------------------------------------------

class Grid:
    """Periodic equidistant grid x_a = a*dx, a = 0..n-1, with an optional
    Bloch twist theta (phase e^{i theta} across one period)."""

    def __init__(self, n, dx, twist=(0.0, 0.0, 0.0)):
        self.n = tuple(int(v) for v in n)            # (nx, ny, nz)
        self.dx = tuple(float(v) for v in dx)
        self.L = tuple(self.n[i] * self.dx[i] for i in range(3))
        self.theta = tuple(float(v) for v in twist)
        self.G = self.n[0] * self.n[1] * self.n[2]
        self.dV = self.dx[0] * self.dx[1] * self.dx[2]
        self.shape = (self.n[2], self.n[1], self.n[0])

    def k(self, j, twisted):
        """Wavenumbers of direction j (0=x, 1=y, 2=z) in FFT order, shaped to
        broadcast against [nz, ny, nx].  The Nyquist index n/2 carries
        -pi/dx.  ``twisted`` adds theta_j / L_j."""
        kj = 2.0 * np.pi * np.fft.fftfreq(self.n[j], d=self.dx[j])
        if twisted:
            kj = kj + self.theta[j] / self.L[j]
        shape = [1, 1, 1]
        shape[2 - j] = self.n[j]
        return kj.reshape(shape)

    def k2(self, twisted):
        return sum(self.k(j, twisted) ** 2 for j in range(3))


def fft3(f):
    return np.fft.fftn(f, axes=AXES3)


def ifft3(f):
    return np.fft.ifftn(f, axes=AXES3)


def deriv(f, j, grid):
    """d_j of a (Bloch-periodic part of a) spinor component:
    IFFT[ i (k_j + theta_j/L_j) FFT[f] ] with the full 3D transform."""
    return ifft3(1j * grid.k(j, True) * fft3(f))


def deriv_real(f, j, grid):
    """d_j of a real periodic field: real part of IFFT[i k_j FFT[f]]."""
    return np.real(ifft3(1j * grid.k(j, False) * fft3(f)))


def laplacian_real(f, grid):
    """Delta f of a real periodic field: real part of IFFT[-|k|^2 FFT[f]]."""
    return np.real(ifft3(-grid.k2(False) * fft3(f)))


def spin(k, psi):
    """(sigma_k psi)_s = sum_t sigma_k[s, t] psi_t, psi shaped [..., 2, z, y, x]."""
    return np.einsum("st,...tzyx->...szyx", SIGMA[k], psi)


def inner(a, b, grid):
    """<a|b> = dV * sum conj(a) b over spin and space (per leading index)."""
    return grid.dV * np.sum(np.conj(a) * b, axis=(-4, -3, -2, -1))


# --------------------------------------------------------------------------
# Single-particle Hamiltonian (Sec. 2.1-2.2; Eq. Schroedinger)
# --------------------------------------------------------------------------

def apply_h(psi, U, B, W, grid):
    """h psi = U psi - sum_j d_j (B d_j psi)
               - (i/2) sum_ijk eps_ijk [ W_i sigma_k d_j psi + d_j (W_i sigma_k psi) ].

    Kinetic (effective mass) term, local potential and the symmetrised
    spin-orbit term W.(-i)(nabla x sigma); U, B real [z,y,x], W real [3,z,y,x]."""
    dpsi = [deriv(psi, j, grid) for j in range(3)]
    h = U * psi
    for j in range(3):
        h = h - deriv(B * dpsi[j], j, grid)
    for i in range(3):
        for j in range(3):
            for k in range(3):
                e = levi_civita(i, j, k)
                if e == 0:
                    continue
                h = h - 0.5j * e * (W[i] * spin(k, dpsi[j])
                                    + deriv(W[i] * spin(k, psi), j, grid))
    return h


def sp_energies(psi, hpsi, grid):
    """eps_alpha = <psi_alpha|h|psi_alpha> and <psi_alpha|h^2|psi_alpha> = ||h psi_alpha||^2."""
    eps = np.real(inner(psi, hpsi, grid))
    hn2 = np.real(inner(hpsi, hpsi, grid))
    return eps, hn2


def convergence_measure(eps_list, hn2_list):
    """Eq. convergence: sqrt( sum_alpha (<h^2> - <h>^2) / sum_alpha 1 ) over all states."""
    eps = np.concatenate(eps_list)
    hn2 = np.concatenate(hn2_list)
    return float(np.sqrt(max(np.sum(hn2 - eps ** 2), 0.0) / eps.size))


# --------------------------------------------------------------------------
# Densities (Eqs. rho, curr, tau; all v^2 = 1)
# --------------------------------------------------------------------------

def densities(psi, grid):
    """rho = sum |psi|^2, tau = sum |d psi|^2,
    J_i = Re sum eps_ijk (-i) psi^dagger sigma_k d_j psi, and div J.
    psi [I, 2, z, y, x].  Returns rho, tau, J[3], divJ."""
    rho = np.sum(np.abs(psi) ** 2, axis=(0, 1))
    dpsi = [deriv(psi, j, grid) for j in range(3)]
    tau = sum(np.sum(np.abs(d) ** 2, axis=(0, 1)) for d in dpsi)
    J = np.zeros((3,) + grid.shape)
    for i in range(3):
        for j in range(3):
            for k in range(3):
                e = levi_civita(i, j, k)
                if e == 0:
                    continue
                J[i] += e * np.real(-1j * np.sum(np.conj(psi) * spin(k, dpsi[j]), axis=(0, 1)))
    divJ = sum(deriv_real(J[i], i, grid) for i in range(3))
    return rho, tau, J, divJ


# --------------------------------------------------------------------------
# Skyrme functional, mean fields, Coulomb, energy (Eq. Skyrme and Sec. 2.2)
# --------------------------------------------------------------------------

def coefficients(p):
    """Isoscalar (T=0) / isovector (T=1) coupling constants from (t, x, W0)."""
    t0, t1, t2, t3 = p["t0"], p["t1"], p["t2"], p["t3"]
    x0, x1, x2, x3 = p["x0"], p["x1"], p["x2"], p["x3"]
    W0 = p["W0"]
    return {
        "rho": (3.0 * t0 / 8.0, -t0 * (0.5 + x0) / 4.0),
        "rhoa": (t3 / 16.0, -t3 * (0.5 + x3) / 24.0),
        "tau": (3.0 * t1 / 16.0 + t2 * (1.25 + x2) / 4.0,
                -t1 * (0.5 + x1) / 8.0 + t2 * (0.5 + x2) / 8.0),
        "drho": (-9.0 * t1 / 64.0 + t2 * (1.25 + x2) / 16.0,
                 3.0 * t1 * (0.5 + x1) / 32.0 + t2 * (0.5 + x2) / 32.0),
        "nJ": (-0.75 * W0, -0.25 * W0),
    }


def _isospin(f):
    """(f_0, f_1) = (f_n + f_p, f_n - f_p)."""
    return (f[0] + f[1], f[0] - f[1])


def _rho0_powers(rho0, alpha):
    safe = rho0 > 1e-30
    r = np.where(safe, rho0, 1.0)
    return np.where(safe, r ** alpha, 0.0), np.where(safe, r ** (alpha - 1.0), 0.0)


def coulomb_potential(rho_p, grid, e2):
    """Poisson in momentum space: V(k) = 4 pi e^2 rho_p(k) / |k|^2, V(0) = 0."""
    k2 = grid.k2(False)
    rk = fft3(rho_p)
    vk = np.zeros_like(rk)
    nz = k2 > 0
    vk[nz] = 4.0 * np.pi * e2 * rk[nz] / k2[nz]
    return np.real(ifft3(vk))


def mean_fields(rho, tau, divJ, p, grid, coulomb):
    """U_q = dE/drho_q, B_q = dE/dtau_q, W_q = dE/dJ_q for q = n (0), p (1).

    rho, tau, divJ are [2, z, y, x].  Returns U[2], B[2], W[2, 3]."""
    C = coefficients(p)
    alpha = p["alpha"]
    rT, tT, dT = _isospin(rho), _isospin(tau), _isospin(divJ)
    lapT = [laplacian_real(rT[T], grid) for T in range(2)]
    gradT = [[deriv_real(rT[T], j, grid) for j in range(3)] for T in range(2)]
    r0a, r0am1 = _rho0_powers(rT[0], alpha)
    U = np.zeros((2,) + grid.shape)
    B = np.zeros((2,) + grid.shape)
    W = np.zeros((2, 3) + grid.shape)
    hb2m = (p["hb2m_n"], p["hb2m_p"])
    for q, s1 in ((0, 1.0), (1, -1.0)):
        s = (1.0, s1)
        for T in range(2):
            U[q] += s[T] * (2.0 * (C["rho"][T] + C["rhoa"][T] * r0a) * rT[T]
                            + C["tau"][T] * tT[T]
                            + 2.0 * C["drho"][T] * lapT[T]
                            + C["nJ"][T] * dT[T])
            U[q] += alpha * r0am1 * C["rhoa"][T] * rT[T] ** 2
            B[q] += s[T] * C["tau"][T] * rT[T]
            for j in range(3):
                W[q, j] -= s[T] * C["nJ"][T] * gradT[T][j]
        B[q] += hb2m[q]
    if coulomb:
        U[1] += coulomb_potential(rho[1], grid, p["e2"])
    return U, B, W


def energy(rho, tau, divJ, p, grid, coulomb):
    """Total energy on the grid (dV * sum of the energy density).

    E = int [ hb2m_n tau_n + hb2m_p tau_p
              + sum_T ( (C_T^rho + C_T^rhoa rho_0^alpha) rho_T^2 + C_T^tau rho_T tau_T
                        + C_T^drho rho_T Delta rho_T + C_T^nJ rho_T div J_T ) ] + E_C,
    E_C = 1/2 int rho_p V_C.  Returns a dict of the parts and the total."""
    C = coefficients(p)
    rT, tT, dT = _isospin(rho), _isospin(tau), _isospin(divJ)
    r0a, _ = _rho0_powers(rT[0], p["alpha"])
    dV = grid.dV
    parts = {
        "kin": dV * np.sum(p["hb2m_n"] * tau[0] + p["hb2m_p"] * tau[1]),
        "rho": 0.0, "tau": 0.0, "drho": 0.0, "nJ": 0.0, "coul": 0.0,
    }
    for T in range(2):
        parts["rho"] += dV * np.sum((C["rho"][T] + C["rhoa"][T] * r0a) * rT[T] ** 2)
        parts["tau"] += dV * np.sum(C["tau"][T] * rT[T] * tT[T])
        parts["drho"] += dV * np.sum(C["drho"][T] * rT[T] * laplacian_real(rT[T], grid))
        parts["nJ"] += dV * np.sum(C["nJ"][T] * rT[T] * dT[T])
    if coulomb:
        parts["coul"] = 0.5 * dV * np.sum(rho[1] * coulomb_potential(rho[1], grid, p["e2"]))
    parts["total"] = sum(parts[k] for k in ("kin", "rho", "tau", "drho", "nJ", "coul"))
    parts["A"] = dV * float(np.sum(rho[0] + rho[1]))
    return parts


# --------------------------------------------------------------------------
# Damped gradient step (Eq. dampstep)
# --------------------------------------------------------------------------

def damped_step(psi, hpsi, eps, grid, hb2m, x0, E0):
    """phi = psi - x0 / (T + E0) (h - eps) psi, with T = hb2m |k + theta/L|^2
    diagonal in momentum space (the FFT of each spin component)."""
    r = hpsi - eps[:, None, None, None, None] * psi
    P = 1.0 / (E0 + hb2m * grid.k2(True))
    return psi - x0 * ifft3(P * fft3(r))


# --------------------------------------------------------------------------
# Matrices, orthonormalisation, diagonalisation, recombination (Sec. 3.3)
# --------------------------------------------------------------------------

def lower_mirror(M):
    """Keep the lower triangle (i >= j) and define the rest by Hermiticity,
    as only i >= j is computed in Fig. 3."""
    L = np.tril(M)
    return L + np.conj(np.tril(M, -1)).T


def overlap(a, b, grid):
    """X_{alpha beta} = <a_alpha | b_beta> (Eqs. normmatrix, hammatrix), lower
    triangle mirrored."""
    A = a.reshape(a.shape[0], -1)
    Bm = b.reshape(b.shape[0], -1)
    return lower_mirror(grid.dV * (np.conj(A) @ Bm.T))


def loewdin(S):
    """C = S^{-1/2} = X Lambda^{-1/2} X^H from the eigendecomposition of S
    (Eq. Loewedin)."""
    lam, X = np.linalg.eigh(S)
    if lam.min() <= 0.0:
        raise np.linalg.LinAlgError("overlap matrix not positive definite")
    return (X * (1.0 / np.sqrt(lam))) @ np.conj(X).T


def rayleigh_ritz(S, H):
    """Exact Rayleigh-Ritz: C = S^{-1/2}, H' = C^H H C = Z Lambda Z^H (ascending),
    M = C Z.  The new states are psi_alpha = sum_beta M_{beta alpha} phi_beta."""
    C = loewdin(S)
    Hp = np.conj(C).T @ H @ C
    Hp = 0.5 * (Hp + np.conj(Hp).T)
    lam, Z = np.linalg.eigh(Hp)
    return C @ Z, lam


def combined_literal(S, H):
    """The paper's combined form (Sec. 3.3.3, Fig. step67): Z from the
    eigendecomposition of H itself (the non-orthonormal basis, H = Z Lambda
    Z^H, ascending), C = S^{-1/2} from the overlap of the same states, and the
    two applied one after the other as one matrix: first the diagonalising
    combination chi_alpha = sum_beta Z_{beta alpha} phi_beta, then Eq.
    orthmatvec with C, psi_alpha = sum_gamma C_{gamma alpha} chi_gamma, i.e.
    M = Z C.  (Reading: the paper's Z^H and C^T act on the column of states;
    with H_ij = <phi_i|h|phi_j> the combination that diagonalises h is Z's
    columns, and C is applied as in Eq. orthmatvec.)  Equal to the exact
    Rayleigh-Ritz step when S = I; otherwise the new states are neither exactly
    orthonormal nor exact Ritz vectors, and the difference vanishes at
    convergence.  The result depends on the phases of Z's columns (fixed as
    below) and, for degenerate eigenvalues of H, on the basis chosen in each
    degenerate space.  Returns (M, Lambda)."""
    Hh = 0.5 * (H + np.conj(H).T)
    lam, Z = np.linalg.eigh(Hh)
    # M = Z C mixes the columns of Z, so the result depends on their phases,
    # which the paper leaves open.  Reading: each eigenvector's largest
    # component (the first one of largest modulus) is made real and positive.
    for k in range(Z.shape[1]):
        i = int(np.argmax(np.abs(Z[:, k])))
        Z[:, k] *= np.conj(Z[i, k]) / abs(Z[i, k])
    return Z @ loewdin(S), lam


def rotate(phi, M):
    """psi_alpha = sum_beta M_{beta alpha} phi_beta (Eq. orthmatvec form)."""
    return np.tensordot(M, phi, axes=(0, 0))


def orthonormalize(psi, grid):
    """Loewdin orthonormalisation of raw states (Eqs. Loewedin, orthmatvec)."""
    return rotate(psi, loewdin(overlap(psi, psi, grid)))


# --------------------------------------------------------------------------
# One iteration (Fig. 1 steps 2-5) and the driver
# --------------------------------------------------------------------------

class State:
    """psi[q], mean fields U, B, W, and the last energy."""

    def __init__(self, psi, U, B, W):
        self.psi = list(psi)
        self.U, self.B, self.W = U, B, W


def initial_state(psi0, grid, p, coulomb, rho0=None, tau0=None):
    """Fig. 1 step 1: orthonormalise the trial states; the mean field comes
    from their densities, or from given initial densities (zero J)."""
    psi = [orthonormalize(psi0[q], grid) for q in range(2)]
    if rho0 is None:
        d = [densities(psi[q], grid) for q in range(2)]
        rho = np.stack([d[q][0] for q in range(2)])
        tau = np.stack([d[q][1] for q in range(2)])
        divJ = np.stack([d[q][3] for q in range(2)])
    else:
        rho, tau = np.asarray(rho0), np.asarray(tau0)
        divJ = np.zeros_like(rho)
    U, B, W = mean_fields(rho, tau, divJ, p, grid, coulomb)
    return State(psi, U, B, W)


def iterate(st, grid, p, coulomb, x0, E0, frozen=False, damping=None, variant="exact"):
    """One damped-gradient iteration.  Mutates ``st`` and returns a record
    with the Ritz values, convergence measure and energy.  ``damping``, if
    given, is a callable (q, U_q, B_q, W_q) -> w [nz,ny,nx] that scales the
    update of the damped step voxel by voxel (phi = psi - w (psi - phi)).
    ``variant`` "exact" (Rayleigh-Ritz in the Loewdin basis) or
    "paper_literal" (the combined form of Sec. 3.3.3, ``combined_literal``).

    Step 2: h psi with h^(n); eps = <psi|h|psi>; phi = psi - x0/(T+E0)(h-eps)psi;
            h phi with the same h^(n).
    Step 3: S = <phi|phi>, H = <phi|h|phi>; Rayleigh-Ritz; psi = phi M.
    Step 4: densities of the new psi; new mean field (unless ``frozen``).
    Step 5: energy."""
    hb2m = (p["hb2m_n"], p["hb2m_p"])
    eps_l, hn2_l, lam_l = [], [], []
    for q in range(2):
        psi = st.psi[q]
        hpsi = apply_h(psi, st.U[q], st.B[q], st.W[q], grid)
        eps, hn2 = sp_energies(psi, hpsi, grid)
        eps_l.append(eps); hn2_l.append(hn2)
        phi = damped_step(psi, hpsi, eps, grid, hb2m[q], x0, E0)
        if damping is not None:
            w = damping(q, st.U[q], st.B[q], st.W[q])
            phi = psi - w[None, None] * (psi - phi)
        hphi = apply_h(phi, st.U[q], st.B[q], st.W[q], grid)
        S = overlap(phi, phi, grid)
        H = overlap(phi, hphi, grid)
        M, lam = rayleigh_ritz(S, H) if variant == "exact" else combined_literal(S, H)
        st.psi[q] = rotate(phi, M)
        lam_l.append(lam)
    d = [densities(st.psi[q], grid) for q in range(2)]
    rho = np.stack([d[q][0] for q in range(2)])
    tau = np.stack([d[q][1] for q in range(2)])
    divJ = np.stack([d[q][3] for q in range(2)])
    if not frozen:
        st.U, st.B, st.W = mean_fields(rho, tau, divJ, p, grid, coulomb)
    E = energy(rho, tau, divJ, p, grid, coulomb)
    return {"lam": lam_l, "eps": eps_l, "delta_eps": convergence_measure(eps_l, hn2_l),
            "E": E["total"], "E_parts": E, "rho": rho, "tau": tau, "divJ": divJ}


def solve(psi0, grid, p, coulomb, x0, E0, maxit, tol, rho0=None, tau0=None,
          frozen=False, callback=None, damping=None, variant="exact"):
    """Iterate until |E_n/A - E_{n-1}/A| < tol (MeV) or maxit iterations."""
    st = initial_state(psi0, grid, p, coulomb, rho0, tau0)
    A = st.psi[0].shape[0] + st.psi[1].shape[0]
    hist = []
    E_prev = None
    for it in range(maxit):
        rec = iterate(st, grid, p, coulomb, x0, E0, frozen=frozen, damping=damping,
                      variant=variant)
        rec["it"] = it
        hist.append({k: rec[k] for k in ("it", "E", "delta_eps")})
        if callback is not None:
            callback(it, rec, st)
        if E_prev is not None and abs(rec["E"] - E_prev) / A < tol:
            return st, rec, hist, True
        E_prev = rec["E"]
    return st, rec, hist, False


def dense_h(U, B, W, grid):
    """The full 2G x 2G matrix of h (columns = h applied to unit vectors),
    for brute-force diagonalisation on tiny grids."""
    nz, ny, nx = grid.shape
    V = 2 * grid.G
    cols = np.zeros((V, V), dtype=np.complex128)
    e = np.zeros((V,), dtype=np.complex128)
    for c in range(V):
        e[:] = 0.0
        e[c] = 1.0
        cols[:, c] = apply_h(e.reshape(2, nz, ny, nx), U, B, W, grid).reshape(-1)
    return cols


def recombination_macs(I, V, combined):
    """Multiply-adds of steps 3d-3e (Sec. 3.3.3): applying C^T then Z^H to
    the I states of length V costs 2 I^2 V; forming the I x I product first
    costs I^3 + I^2 V.  Counted by the loop structure of each variant."""
    macs = 0
    if combined:
        for _ in range(I):          # I x I times I x I
            for _ in range(I):
                macs += I
        for _ in range(I):          # I x I times I x V
            macs += I * V
    else:
        for _ in range(2):          # two I x I times I x V products
            for _ in range(I):
                macs += I * V
    return macs
