"""Pins of the oracle's matrices, orthonormalisation, Rayleigh-Ritz,
recombination and whole iteration (CPU only)."""
import os

import numpy as np
import pytest
import scipy.linalg

import oracle as O
from paper_1610_07522_gb300 import inputs as IN

P = dict(IN.SLY4)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small_states(grid, I, rng):
    return IN.random_superpositions(grid.n, grid.dx, I, rng) / 7.0


def test_overlap_matches_bruteforce_loops():
    rng = np.random.default_rng(1)
    grid = O.Grid((4, 2, 2), (1.0, 1.0, 1.3))
    a = IN.random_spinors(grid.n, 3, rng)
    b = IN.random_spinors(grid.n, 3, rng)
    X = O.overlap(a, b, grid)
    fa, fb = a.reshape(3, -1), b.reshape(3, -1)
    for i in range(3):
        for j in range(3):
            if i >= j:   # only the lower triangle is computed (Fig. 3)
                want = 0.0
                for v in range(fa.shape[1]):
                    want += np.conj(fa[i, v]) * fb[j, v]
                assert abs(X[i, j] - grid.dV * want) < 1e-12
            else:
                assert X[i, j] == np.conj(X[j, i])


def test_loewdin_properties():
    rng = np.random.default_rng(2)
    grid = O.Grid((6, 6, 6), (1.0, 1.0, 1.0))
    phi = _small_states(grid, 6, rng)
    S = O.overlap(phi, phi, grid)
    C = O.loewdin(S)
    assert np.allclose(C, C.conj().T, atol=1e-12)
    assert np.allclose(C.conj().T @ S @ C, np.eye(6), atol=1e-11)
    psi = O.rotate(phi, C)
    assert np.allclose(O.overlap(psi, psi, grid), np.eye(6), atol=1e-11)
    # Loewdin states are the orthonormal set closest to phi (least squares):
    # any other orthonormal basis of the span is farther away.
    d0 = np.sum(np.abs(psi - phi) ** 2)
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6)))
    other = O.rotate(psi, Q.T)
    assert np.sum(np.abs(other - phi) ** 2) > d0


def test_rayleigh_ritz_matches_generalised_eigenproblem_and_cholesky():
    rng = np.random.default_rng(3)
    grid = O.Grid((6, 6, 6), (1.0, 1.0, 1.0))
    phi = _small_states(grid, 5, rng)
    U = IN.random_smooth_field(grid.n, rng, -40.0, 10.0)
    B = IN.random_smooth_field(grid.n, rng, 20.0, 5.0)
    W = np.stack([IN.random_smooth_field(grid.n, rng, 0.0, 5.0) for _ in range(3)])
    hphi = O.apply_h(phi, U, B, W, grid)
    S = O.overlap(phi, phi, grid)
    H = O.overlap(phi, hphi, grid)
    M, lam = O.rayleigh_ritz(S, H)
    ref = scipy.linalg.eigh(H, S, eigvals_only=True)
    assert np.allclose(lam, ref, atol=1e-10 * np.max(np.abs(ref)))
    assert np.allclose(M.conj().T @ S @ M, np.eye(5), atol=1e-11)
    assert np.allclose(M.conj().T @ H @ M, np.diag(lam), atol=1e-9)
    # Cholesky route: S = L L^H, eig(L^-1 H L^-H) -> same values and projector
    Lc = np.linalg.cholesky(S)
    Li = np.linalg.inv(Lc)
    lam2, Z2 = np.linalg.eigh(Li @ H @ Li.conj().T)
    M2 = Li.conj().T @ Z2
    assert np.allclose(lam, lam2, atol=1e-12 * np.max(np.abs(lam)))
    P1 = O.rotate(phi, M).reshape(5, -1)
    P2 = O.rotate(phi, M2).reshape(5, -1)
    probe = rng.standard_normal(P1.shape[1])
    proj = lambda Q: Q.T @ (np.conj(Q) @ probe)
    assert np.allclose(proj(P1), proj(P2), atol=1e-10)


def test_rotate_matches_bruteforce():
    rng = np.random.default_rng(4)
    phi = IN.random_spinors((2, 2, 2), 3, rng)
    M = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    out = O.rotate(phi, M)
    for a in range(3):
        want = sum(M[b, a] * phi[b] for b in range(3))
        assert np.allclose(out[a], want, atol=1e-13)


def test_recombination_cost_matches_paper():
    """Sec. 3.3.3: combining the two I x I factors first reduces the
    multiply-adds from 2 I^2 V to I^3 + I^2 V (fixture cites the passage)."""
    with open(os.path.join(GOLDEN, "recombination_cost.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for I, V, sep, comb in rows:
        I, V, sep, comb = int(I), int(V), int(sep), int(comb)
        assert O.recombination_macs(I, V, combined=False) == sep
        assert O.recombination_macs(I, V, combined=True) == comb


def _fermi_gas(grid, Nn, Np):
    labs = [IN.plane_wave_labels(grid.n, grid.dx, I) for I in (Nn, Np)]
    return [IN.plane_wave_states(grid.n, grid.dx, l) for l in labs], labs


def test_free_fermi_gas_closed_form_and_fixed_point():
    """Closed shells (14 n + 38 p on 8^3): uniform rho_q = I_q/V,
    tau_q = sum |k|^2 / V, J = 0; the energy is the uniform-matter
    functional times V; eps = B_q |k|^2 + U_q; one iteration is a fixed point."""
    grid = O.Grid((8, 8, 8), (1.0, 1.0, 1.0))
    psi, labs = _fermi_gas(grid, 14, 38)
    vol = 512.0
    st = O.initial_state(psi, grid, P, coulomb=False)
    for q, I in ((0, 14), (1, 38)):
        ks = [np.array(l[:3]) * 2 * np.pi / 8 for l in labs[q]]
        rho, tau, J, divJ = O.densities(st.psi[q], grid)
        assert np.allclose(rho, I / vol, atol=1e-14)
        assert np.allclose(tau, sum(k.dot(k) for k in ks) / vol, atol=1e-13)
        assert np.max(np.abs(J)) < 1e-14
    rec0 = O.iterate(st, grid, P, False, 0.45, 100.0)
    rho_n, rho_p = 14 / vol, 38 / vol
    t = [sum((np.array(l[:3]) * 2 * np.pi / 8).dot(np.array(l[:3]) * 2 * np.pi / 8) for l in labs[q]) / vol for q in range(2)]
    C = O.coefficients(P)
    r = (rho_n + rho_p, rho_n - rho_p); tt = (t[0] + t[1], t[0] - t[1])
    e = P["hb2m_n"] * t[0] + P["hb2m_p"] * t[1]
    for T in range(2):
        e += (C["rho"][T] + C["rhoa"][T] * r[0] ** P["alpha"]) * r[T] ** 2 + C["tau"][T] * r[T] * tt[T]
    assert abs(rec0["E"] - e * vol) < 1e-11 * abs(e * vol)
    for q in range(2):
        ks2 = sorted((np.array(l[:3]) * 2 * np.pi / 8).dot(np.array(l[:3]) * 2 * np.pi / 8) for l in labs[q])
        want = np.sort(st.B[q].flat[0] * np.array(ks2) + st.U[q].flat[0])
        assert np.allclose(np.sort(rec0["lam"][q]), want, atol=1e-10)
    rec1 = O.iterate(st, grid, P, False, 0.45, 100.0)
    assert abs(rec1["E"] - rec0["E"]) < 1e-12 * abs(rec0["E"])
    assert rec1["delta_eps"] < 1e-9


def test_frozen_mean_field_converges_to_dense_eigenvalues():
    """8^3 grid, fixed smooth U, B, W: the damped-gradient iteration with
    Rayleigh-Ritz converges to the I lowest eigenvalues of the dense 1024 x 1024 h."""
    rng = np.random.default_rng(5)
    grid = O.Grid((8, 8, 8), (1.0, 1.0, 1.0))
    U = IN.random_smooth_field(grid.n, rng, -30.0, 25.0)
    B = IN.random_smooth_field(grid.n, rng, 20.0, 4.0)
    W = np.stack([IN.random_smooth_field(grid.n, rng, 0.0, 6.0) for _ in range(3)])
    ev = np.linalg.eigvalsh(O.dense_h(U, B, W, grid))
    I = int(np.argmax(np.diff(ev[:12])[1:])) + 2   # occupy up to the largest low gap
    assert ev[I] - ev[I - 1] > 0.3
    psi0 = IN.noisy_plane_waves(grid.n, grid.dx, I, 0.1, rng)
    st = O.State([O.orthonormalize(psi0, grid)] * 2, np.stack([U, U]), np.stack([B, B]), np.stack([W, W]))
    for it in range(600):
        rec = O.iterate(st, grid, P, False, 0.45, 100.0, frozen=True)
    assert np.max(np.abs(np.sort(rec["lam"][0]) - ev[:I])) < 1e-9


def test_self_consistent_aufbau():
    """At self-consistency the occupied levels are the lowest eigenvalues of
    the dense h built from the converged densities (2 n + 2 p that bind into
    a droplet in a 6^3 box; Ritz values converge quadratically in the residual)."""
    w = IN.Workload(name="aufbau", grid=(6, 6, 6), dx=(1.0, 1.0, 1.0), N=2, Z=2, seed=1, noise=0.1)
    grid = O.Grid(w.grid, w.dx)
    inp = IN.make_inputs(w)
    st, rec, hist, conv = O.solve(inp["psi0"], grid, P, False, w.x0, w.E0, maxit=450, tol=1e-15)
    assert rec["delta_eps"] < 1e-3
    assert rec["E"] < hist[0]["E"] - 5.0     # the droplet is bound below the start
    for q in range(2):
        ev = np.linalg.eigvalsh(O.dense_h(st.U[q], st.B[q], st.W[q], grid))
        occ = np.sort(rec["lam"][q])
        assert np.max(np.abs(occ - ev[:occ.size])) < 1e-4
        assert ev[occ.size] > occ[-1] + 1.0    # no empty level below the Fermi level


def test_random_superpositions_are_plane_wave_sums():
    """The k-space synthesis equals the explicit sum of the 2I lowest spin
    plane waves with the same seeded coefficients."""
    import numpy as np
    from paper_1610_07522_gb300 import inputs as IN
    grid, dx, I = (8, 12, 10), (1.0, 0.9, 1.1), 9
    got = IN.random_superpositions(grid, dx, I, np.random.default_rng(5))
    rng = np.random.default_rng(5)
    basis = IN.plane_wave_states(grid, dx, IN.plane_wave_labels(grid, dx, 2 * I))
    c = rng.standard_normal((I, 2 * I)) + 1j * rng.standard_normal((I, 2 * I))
    want = np.tensordot(c, basis, axes=(1, 0))
    assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want))


def _herm(rng, n, scale=1.0):
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return scale * (A + A.conj().T) / 2


def test_combined_literal_equals_exact_ritz_for_orthonormal_states():
    import numpy as np
    from oracle import sky_oracle as O
    rng = np.random.default_rng(31)
    n = 9
    H = _herm(rng, n, 10.0)
    M1, l1 = O.combined_literal(np.eye(n), H)
    M2, l2 = O.rayleigh_ritz(np.eye(n), H)
    assert np.max(np.abs(l1 - l2)) < 1e-12
    # same vectors up to a phase per column (distinct eigenvalues)
    ov = np.abs(np.sum(np.conj(M1) * M2, axis=0))
    assert np.max(np.abs(ov - 1.0)) < 1e-12
    # the phase convention: largest component of each column real and positive
    for k in range(n):
        i = int(np.argmax(np.abs(M1[:, k])))
        assert abs(M1[i, k].imag) < 1e-14 and M1[i, k].real > 0


def test_combined_literal_differs_at_first_order_in_the_overlap():
    """With S = I + eps E the literal form is neither orthonormal nor exact:
    both defects are first order in eps (and vanish with it)."""
    import numpy as np
    from oracle import sky_oracle as O
    rng = np.random.default_rng(32)
    n = 8
    H = np.diag(np.arange(n) * 3.0) + _herm(rng, n, 0.5)
    E = _herm(rng, n, 1.0)
    defects = []
    for eps in (1e-2, 1e-3):
        S = np.eye(n) + eps * E
        M, lam = O.combined_literal(S, H)
        Mx, lx = O.rayleigh_ritz(S, H)
        ortho = np.max(np.abs(M.conj().T @ S @ M - np.eye(n)))
        assert np.max(np.abs(Mx.conj().T @ S @ Mx - np.eye(n))) < 1e-12
        defects.append((ortho, np.max(np.abs(lam - lx))))
    for k in range(2):
        assert defects[0][k] > 1e-6
        ratio = defects[0][k] / defects[1][k]
        assert 5.0 < ratio < 20.0          # linear in eps


def test_literal_iteration_keeps_the_fixed_point():
    """Exact eigenstates of a frozen h are a fixed point of the literal variant."""
    import numpy as np
    from oracle import sky_oracle as O
    from paper_1610_07522_gb300 import inputs as IN
    rng = np.random.default_rng(33)
    g = O.Grid((4, 4, 4), (1.0, 1.0, 1.0))
    p = dict(IN.SLY4)
    U = np.stack([rng.uniform(-40, 0, g.shape) for _ in range(2)])
    Bf = np.stack([20.7 + rng.uniform(0, 3, g.shape) for _ in range(2)])
    Wf = np.stack([rng.uniform(-1, 1, (3,) + g.shape) for _ in range(2)])
    psi, lams = [], []
    for q in range(2):
        Hd = O.dense_h(U[q], Bf[q], Wf[q], g)
        lam, vec = np.linalg.eigh(0.5 * (Hd + Hd.conj().T))
        psi.append((vec[:, :4].T / np.sqrt(g.dV)).reshape((4, 2) + g.shape))
        lams.append(lam[:4])
    st = O.State(psi, U, Bf, Wf)
    rec = O.iterate(st, g, p, False, 0.45, 100.0, frozen=True, variant="paper_literal")
    for q in range(2):
        assert np.max(np.abs(rec["lam"][q] - lams[q])) < 1e-9
