"""Parity of every libsky entry point with the FP64 CPU oracle (GPU).

All inputs come from the seeded generators; both sides receive the same
arrays.  Tolerances (FP64 form): per-call results element by element within
1e-12 of the largest magnitude (FFT and GEMM rounding, a few ulp times
log N growth); single-particle energies within 1e-9 MeV and total energies
within 1e-10 relative, as stated for the FP64 form.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_1610_07522_gb300 import binding as B
from paper_1610_07522_gb300 import inputs as IN

pytestmark = pytest.mark.gpu

P = dict(IN.SLY4)
REL = 1e-12


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def relerr(got, want):
    return float(np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300))


class Ctx:
    def __init__(self, grid, dx=(1.0, 1.0, 1.0), twist=(0.0, 0.0, 0.0), coulomb=False,
                 max_states=64, prec=B.SKY_F64):
        self.grid = O.Grid(grid, dx, twist)
        self.ctx = B.sky_init(grid, dx, P, coulomb, twist, prec, max_states,
                              torch.cuda.current_stream().cuda_stream)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        B.sky_sync(self.ctx)
        B.sky_destroy(self.ctx)


CASES = [
    ((8, 8, 8), (1.0, 1.0, 1.0), (0.0, 0.0, 0.0)),
    ((16, 16, 16), (1.0, 1.0, 1.0), (0.0, 0.0, 0.0)),
    ((24, 24, 24), (1.0, 1.0, 1.0), (0.0, 0.0, 0.0)),
    ((12, 16, 20), (0.9, 1.1, 1.0), (0.3, -1.2, 2.0)),
    ((32, 8, 24), (1.0, 1.0, 1.0), (-2.0, 0.5, 0.0)),
]


def _fields(grid, rng):
    U = IN.random_smooth_field(grid.n, rng, -40.0, 30.0)
    Bf = IN.random_smooth_field(grid.n, rng, 20.0, 6.0)
    W = np.stack([IN.random_smooth_field(grid.n, rng, 0.0, 10.0) for _ in range(3)])
    return U, Bf, W


@pytest.mark.parametrize("case", CASES)
def test_apply_h(case):
    rng = np.random.default_rng(1)
    with Ctx(*case) as c:
        g = c.grid
        I = 5
        psi = IN.random_spinors(g.n, I, rng)
        U, Bf, W = _fields(g, rng)
        want = O.apply_h(psi, U, Bf, W, g)
        eps_w, hn2_w = O.sp_energies(psi, want, g)
        d_psi, d_h = dev(psi), torch.zeros(psi.shape, dtype=torch.complex128, device="cuda:0")
        eps, hn2 = torch.zeros(I, dtype=torch.float64, device="cuda:0"), torch.zeros(I, dtype=torch.float64, device="cuda:0")
        B.sky_apply_h(c.ctx, dev(U), dev(Bf), dev(W), d_psi, d_h, I, eps, hn2)
        B.sky_sync(c.ctx)
        assert relerr(host(d_h), want) < REL
        assert relerr(host(eps), eps_w) < REL
        assert relerr(host(hn2), hn2_w) < REL


def test_apply_h_ragged_chunks(monkeypatch):
    """Scratch limited to 1 MiB: the 16^3 states run in chunks of 2, 2, 2, 1."""
    monkeypatch.setenv("SKY_SCRATCH_MB", "1")
    rng = np.random.default_rng(2)
    with Ctx((16, 16, 16), twist=(0.2, 0.4, -0.6)) as c:
        g = c.grid
        I = 7
        psi = IN.random_spinors(g.n, I, rng)
        U, Bf, W = _fields(g, rng)
        want = O.apply_h(psi, U, Bf, W, g)
        d_h = torch.zeros(psi.shape, dtype=torch.complex128, device="cuda:0")
        eps = torch.zeros(I, dtype=torch.float64, device="cuda:0")
        B.sky_apply_h(c.ctx, dev(U), dev(Bf), dev(W), dev(psi), d_h, I, eps, None)
        assert relerr(host(d_h), want) < REL
        assert relerr(host(eps), O.sp_energies(psi, want, g)[0]) < REL
        rho_w, tau_w, J_w, dJ_w = O.densities(psi, g)
        rho, tau = torch.zeros(g.G, dtype=torch.float64, device="cuda:0"), torch.zeros(g.G, dtype=torch.float64, device="cuda:0")
        J, dJ = torch.zeros(3 * g.G, dtype=torch.float64, device="cuda:0"), torch.zeros(g.G, dtype=torch.float64, device="cuda:0")
        B.sky_densities(c.ctx, dev(psi), I, rho, tau, J, dJ)
        assert relerr(host(rho), rho_w.ravel()) < REL
        assert relerr(host(tau), tau_w.ravel()) < REL
        assert relerr(host(J), J_w.ravel()) < REL


@pytest.mark.parametrize("case", CASES[1:4])
def test_damped_step(case):
    rng = np.random.default_rng(3)
    with Ctx(*case) as c:
        g = c.grid
        I = 3
        psi = IN.random_spinors(g.n, I, rng)
        hpsi = IN.random_spinors(g.n, I, rng) * 30.0
        eps = rng.uniform(-40, 10, I)
        for q in (0, 1):
            want = O.damped_step(psi, hpsi, eps, g, P["hb2m_n" if q == 0 else "hb2m_p"], 0.45, 100.0)
            phi = torch.zeros(psi.shape, dtype=torch.complex128, device="cuda:0")
            B.sky_damped_step(c.ctx, q, dev(psi), dev(hpsi), dev(eps), phi, I, 0.45, 100.0)
            assert relerr(host(phi), want) < REL
        # a second E0 rebuilds the cached preconditioner table
        want = O.damped_step(psi, hpsi, eps, g, P["hb2m_n"], 0.3, 60.0)
        phi = torch.zeros(psi.shape, dtype=torch.complex128, device="cuda:0")
        B.sky_damped_step(c.ctx, 0, dev(psi), dev(hpsi), dev(eps), phi, I, 0.3, 60.0)
        assert relerr(host(phi), want) < REL


@pytest.mark.parametrize("I", [1, 2, 31, 37, 70])
def test_overlap(I):
    rng = np.random.default_rng(4 + I)
    with Ctx((16, 16, 16), max_states=80) as c:
        g = c.grid
        a = IN.random_spinors(g.n, I, rng)
        b = IN.random_spinors(g.n, I, rng)
        X = torch.zeros((I, I), dtype=torch.complex128, device="cuda:0")
        B.sky_overlap(c.ctx, dev(a), dev(b), I, X)
        assert relerr(host(X), O.overlap(a, b, g)) < REL
        B.sky_overlap(c.ctx, dev(a), dev(a), I, X)
        assert relerr(host(X), O.overlap(a, a, g)) < REL


def _phi_h(g, I, rng):
    phi = IN.random_superpositions(g.n, g.dx, I, rng) / np.sqrt(g.L[0] * g.L[1] * g.L[2]) * 3
    U, Bf, W = _fields(g, rng)
    return phi, O.apply_h(phi, U, Bf, W, g)


@pytest.mark.parametrize("I", [1, 2, 5, 16, 33])
def test_loewdin_and_rayleigh_ritz(I):
    rng = np.random.default_rng(10 + I)
    with Ctx((16, 16, 16)) as c:
        g = c.grid
        phi, hphi = _phi_h(g, I, rng)
        S, H = O.overlap(phi, phi, g), O.overlap(phi, hphi, g)
        C_w = O.loewdin(S)
        M_w, lam_w = O.rayleigh_ritz(S, H)
        dS, dH = dev(S), dev(H)
        C = torch.zeros_like(dS)
        M = torch.zeros_like(dS)
        lam = torch.zeros(I, dtype=torch.float64, device="cuda:0")
        B.sky_orthonormalize(c.ctx, dS, I, C)
        B.sky_subspace_diag(c.ctx, dH, C, I, M, lam)
        B.sky_sync(c.ctx)
        Cg, Mg, lg = host(C), host(M), host(lam)
        assert relerr(Cg, C_w) < 1e-11
        assert np.max(np.abs(lg - lam_w)) < 1e-9
        assert np.max(np.abs(Mg.conj().T @ S @ Mg - np.eye(I))) < 1e-11
        assert np.max(np.abs(Mg.conj().T @ H @ Mg - np.diag(lam_w))) < 1e-9 * max(1.0, np.max(np.abs(lam_w)))
        # Ritz vectors agree up to a phase per (non-degenerate) column
        for j in range(I):
            k = int(np.argmax(np.abs(M_w[:, j])))
            ph = Mg[k, j] / M_w[k, j]
            assert abs(abs(ph) - 1) < 1e-9
            assert np.max(np.abs(Mg[:, j] - ph * M_w[:, j])) < 1e-8 * np.max(np.abs(M_w[:, j]))


def test_rotate():
    rng = np.random.default_rng(5)
    for I in (1, 3, 40):
        with Ctx((16, 16, 16)) as c:
            phi = IN.random_spinors(c.grid.n, I, rng)
            M = rng.standard_normal((I, I)) + 1j * rng.standard_normal((I, I))
            out = torch.zeros(phi.shape, dtype=torch.complex128, device="cuda:0")
            B.sky_rotate(c.ctx, dev(phi), dev(M), I, out)
            assert relerr(host(out), O.rotate(phi, M)) < REL


@pytest.mark.parametrize("case", CASES[1:])
def test_densities(case):
    rng = np.random.default_rng(6)
    with Ctx(*case) as c:
        g = c.grid
        I = 9
        psi = O.orthonormalize(IN.random_superpositions(g.n, g.dx, I, rng), g)
        rho_w, tau_w, J_w, dJ_w = O.densities(psi, g)
        z = lambda n: torch.zeros(n, dtype=torch.float64, device="cuda:0")
        rho, tau, J, dJ = z(g.G), z(g.G), z(3 * g.G), z(g.G)
        B.sky_densities(c.ctx, dev(psi), I, rho, tau, J, dJ)
        assert relerr(host(rho), rho_w.ravel()) < REL
        assert relerr(host(tau), tau_w.ravel()) < REL
        assert relerr(host(J), J_w.ravel()) < REL
        assert relerr(host(dJ), dJ_w.ravel()) < 1e-11
        B.sky_densities(c.ctx, dev(psi), I, rho, tau, None, dJ)
        assert relerr(host(dJ), dJ_w.ravel()) < 1e-11
        B.sky_densities(c.ctx, dev(psi), 0, rho, tau, J, dJ)     # no states: zero fields
        assert np.all(host(rho) == 0) and np.all(host(dJ) == 0)


@pytest.mark.parametrize("coulomb", [False, True])
@pytest.mark.parametrize("case", [CASES[2], CASES[3]])
def test_mean_fields_and_energy(case, coulomb):
    rng = np.random.default_rng(7)
    with Ctx(*case, coulomb=coulomb) as c:
        g = c.grid
        ds = [O.densities(O.orthonormalize(IN.random_superpositions(g.n, g.dx, I, rng), g), g) for I in (6, 4)]
        rho = np.stack([d[0] for d in ds]); tau = np.stack([d[1] for d in ds]); dJ = np.stack([d[3] for d in ds])
        U_w, B_w, W_w = O.mean_fields(rho, tau, dJ, P, g, coulomb)
        E_w = O.energy(rho, tau, dJ, P, g, coulomb)
        U = torch.zeros((2, g.G), dtype=torch.float64, device="cuda:0")
        Bf = torch.zeros_like(U)
        W = torch.zeros((2, 3, g.G), dtype=torch.float64, device="cuda:0")
        out = torch.zeros(8, dtype=torch.float64, device="cuda:0")
        B.sky_mean_fields(c.ctx, dev(rho), dev(tau), dev(dJ), U, Bf, W)
        B.sky_energy(c.ctx, dev(rho), dev(tau), dev(dJ), out)
        B.sky_sync(c.ctx)
        assert relerr(host(U), U_w.reshape(2, -1)) < 1e-11
        assert relerr(host(Bf), B_w.reshape(2, -1)) < REL
        assert relerr(host(W), W_w.reshape(2, 3, -1)) < 1e-11
        e = host(out)
        keys = ["total", "kin", "rho", "tau", "drho", "nJ", "coul", "A"]
        for i, k in enumerate(keys):
            assert abs(e[i] - E_w[k]) <= 1e-11 * max(1.0, abs(E_w[k])), (k, e[i], E_w[k])


def test_sp_spread():
    rng = np.random.default_rng(8)
    eps = rng.uniform(-50, 0, 400)
    hn2 = eps ** 2 + rng.uniform(0, 3, 400)
    with Ctx((8, 8, 8)) as c:
        out = torch.zeros(2, dtype=torch.float64, device="cuda:0")
        B.sky_sp_spread(c.ctx, dev(eps), dev(hn2), 400, out)
        got = host(out)
    assert abs(got[0] - O.convergence_measure([eps], [hn2])) < 1e-12 * got[0]
    assert abs(got[1] - eps.sum()) < 1e-12 * abs(eps.sum())


def test_status_reporting():
    with Ctx((8, 8, 8), max_states=4) as c:
        # I beyond max_states is refused before anything is enqueued
        X = torch.zeros((5, 5), dtype=torch.complex128, device="cuda:0")
        with pytest.raises(B.SkyError) as ei:
            B.sky_overlap(c.ctx, X, X, 5, X)
        assert ei.value.status == B.SKY_EINVAL
        with pytest.raises(B.SkyError):
            B.sky_rotate(c.ctx, X, X, 2, X)            # output aliases input
        # I == 0 is a no-op
        B.sky_apply_h(c.ctx, X, X, X, X, X.view(-1)[1:], 0)
        # two identical states: overlap singular -> SKY_ENOTPD from the device
        S = dev(np.array([[1.0, 1.0], [1.0, 1.0]], dtype=complex))
        C = torch.zeros_like(S)
        B.sky_orthonormalize(c.ctx, S, 2, C)
        with pytest.raises(B.SkyError) as ei:
            B.sky_sync(c.ctx)
        assert ei.value.status == B.SKY_ENOTPD
        B.sky_sync(c.ctx)                              # status word cleared


def _gpu_run(w, inp, nit):
    from paper_1610_07522_gb300.solver import Solver
    s = Solver(w, prec=B.SKY_F64)
    s.load(inp["psi0"], inp.get("rho0"), inp.get("tau0"))
    recs = []
    for _ in range(nit):
        s.step()
        E, de, parts = s.energy()
        lam = host(s.lam)
        recs.append({"E": E, "delta_eps": de, "lam": [np.sort(lam[:w.N]), np.sort(lam[w.N:])],
                     "rho": host(s.rho).copy()})
    s.close()
    return recs


def _oracle_run(w, inp, nit):
    g = O.Grid(w.grid, w.dx, w.twist)
    st = O.initial_state(inp["psi0"], g, w.params, w.coulomb, inp.get("rho0"), inp.get("tau0"))
    return [O.iterate(st, g, w.params, w.coulomb, w.x0, w.E0) for _ in range(nit)]


def _compare_runs(gpu, ora, e_rel=1e-10, lam_abs=1e-9, rho_rel=1e-10):
    for k, (a, b) in enumerate(zip(gpu, ora)):
        assert abs(a["E"] - b["E"]) <= e_rel * abs(b["E"]), (k, a["E"], b["E"])
        assert abs(a["delta_eps"] - b["delta_eps"]) <= 1e-8 * max(1.0, b["delta_eps"]), k
        for q in range(2):
            assert np.max(np.abs(a["lam"][q] - np.sort(b["lam"][q]))) < lam_abs, k
        assert relerr(a["rho"], b["rho"].reshape(2, -1)) < rho_rel, k


def test_iterations_16cubed_16n16p():
    """The 16^3, 16 n + 16 p workload: 12 full iterations against the oracle."""
    w = IN.WORKLOADS["sly4_16cubed_16n16p_fp64"]
    inp = IN.make_inputs(w)
    _compare_runs(_gpu_run(w, inp, 12), _oracle_run(w, inp, 12))


def test_iterations_16cubed_16n16p_whole_run():
    """The 16^3, 16 n + 16 p workload for its whole iteration budget (300)
    against the oracle, iteration by iteration.  The two trajectories do not
    part: measured over 800 iterations on a GB300, the total energies agree to
    8.5e-13 relative and the Ritz values to 6e-11 MeV at worst (1.5e-13 and
    2.1e-12 MeV within the first 300); the bounds below leave a factor 10-50.
    The run does not meet the 1e-6 MeV stop rule within its budget (the gas
    keeps clustering; |dE/A| has a minimum of 3.4e-6 MeV near iteration 60),
    so the comparison covers the whole path the method takes."""
    w = IN.WORKLOADS["sly4_16cubed_16n16p_fp64"]
    inp = IN.make_inputs(w)
    gpu = _gpu_run(w, inp, w.maxit)
    ora = _oracle_run(w, inp, w.maxit)
    _compare_runs(gpu, ora, e_rel=1e-11, lam_abs=1e-10, rho_rel=1e-10)


def test_iterations_twisted_coulomb_small():
    w = IN.Workload(name="t", grid=(12, 16, 8), dx=(1.0, 0.9, 1.2), N=9, Z=7, coulomb=True,
                    twist=(1.0, -0.5, 2.2), init="blobs", seed=33)
    inp = IN.make_inputs(w)
    _compare_runs(_gpu_run(w, inp, 6), _oracle_run(w, inp, 6))


def test_iterations_24cubed_280n120p_coulomb():
    """The full-size 24^3, 280 n + 120 p Coulomb workload: 2 iterations (the
    oracle takes ~30 s per iteration)."""
    w = IN.WORKLOADS["sly4_24cubed_280n120p_coulomb_fp64"]
    inp = IN.make_inputs(w)
    _compare_runs(_gpu_run(w, inp, 2), _oracle_run(w, inp, 2))


@pytest.mark.parametrize("eta", [1e-3, 0.02, 0.5, 15.0])
def test_loewdin_both_routes(eta):
    """Near-orthonormal states (||S - I||_F < 1/2: Newton-Schulz route) and
    strongly non-orthonormal ones (eigendecomposition route) give the oracle's
    S^{-1/2}."""
    rng = np.random.default_rng(int(eta * 1e4))
    with Ctx((16, 16, 16)) as c:
        g = c.grid
        I = 40
        psi = O.orthonormalize(IN.random_superpositions(g.n, g.dx, I, rng), g)
        phi = psi + eta * IN.random_superpositions(g.n, g.dx, I, rng) / np.sqrt(g.L[0] ** 3) / 10
        S = O.overlap(phi, phi, g)
        C = torch.zeros((I, I), dtype=torch.complex128, device="cuda:0")
        B.sky_orthonormalize(c.ctx, dev(S), I, C)
        B.sky_sync(c.ctx)
        Cg = host(C)
        assert relerr(Cg, O.loewdin(S)) < 1e-11
        assert np.max(np.abs(Cg.conj().T @ S @ Cg - np.eye(I))) < 1e-11


# ------------------------------------------------------------------ FP32 form
# Spinors stored as complex64 with FP32 FFTs; matrices, reductions and fields
# FP64.  The oracle runs in FP64 on the same FP32-rounded inputs, so the
# differences are the kernels' FP32 arithmetic only.  FFT-based results:
# within 4e-6 of the largest magnitude (single-precision rounding times the
# log2 n passes of each transform); the overlap as exact split products of
# four 8-bit digits per value (digits to 2^-32 of each row's scale): 1e-8;
# the recombined states are stored in FP32: 1e-6.
REL32 = 4e-6


def _r32(a):
    return a.astype(np.complex64).astype(np.complex128)


def dev32(a):
    return torch.from_numpy(np.ascontiguousarray(a.astype(np.complex64))).to("cuda:0")


@pytest.mark.parametrize("case", [CASES[2], CASES[3], ((32, 32, 32), (1.0, 1.0, 1.0), (0.5, 0.0, -0.5)),
                                  ((64, 48, 16), (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))])
def test_fp32_apply_h_damped_densities(case):
    rng = np.random.default_rng(21)
    with Ctx(*case, prec=B.SKY_F32) as c:
        g = c.grid
        I = 3
        psi = _r32(IN.random_spinors(g.n, I, rng))
        U, Bf, W = _fields(g, rng)
        want = O.apply_h(psi, U, Bf, W, g)
        d_h = torch.zeros(psi.shape, dtype=torch.complex64, device="cuda:0")
        eps = torch.zeros(I, dtype=torch.float64, device="cuda:0")
        B.sky_apply_h(c.ctx, dev(U), dev(Bf), dev(W), dev32(psi), d_h, I, eps, None)
        assert relerr(host(d_h), want) < REL32
        assert relerr(host(eps), O.sp_energies(psi, want, g)[0]) < REL32
        hpsi = _r32(want)
        e = rng.uniform(-40, 10, I)
        phi = torch.zeros(psi.shape, dtype=torch.complex64, device="cuda:0")
        B.sky_damped_step(c.ctx, 1, dev32(psi), dev32(hpsi), dev(e), phi, I, 0.45, 100.0)
        assert relerr(host(phi), O.damped_step(psi, hpsi, e, g, P["hb2m_p"], 0.45, 100.0)) < REL32
        z = lambda n: torch.zeros(n, dtype=torch.float64, device="cuda:0")
        rho, tau, J, dJ = z(g.G), z(g.G), z(3 * g.G), z(g.G)
        B.sky_densities(c.ctx, dev32(psi), I, rho, tau, J, dJ)
        rw, tw, Jw, dJw = O.densities(psi, g)
        assert relerr(host(rho), rw.ravel()) < REL32
        assert relerr(host(tau), tw.ravel()) < REL32
        assert relerr(host(J), Jw.ravel()) < REL32


@pytest.mark.parametrize("grid,twist,I", [((12, 16, 20), (0.3, -0.8, 1.7), 37),
                                           ((24, 24, 24), (0.0, 0.0, 0.0), 5),
                                           ((24, 24, 24), (1.3, -0.2, 0.9), 120),
                                           ((32, 8, 12), (-2.1, 0.4, 3.0), 9)])
def test_fp32_fused_h_matches_general_path_and_oracle(grid, twist, I):
    """The FP32 forms' h psi in one fused pass per axis (the default for axis
    lengths up to 24) against the general gradient / local / divergence
    passes (knob 0) and the oracle, with <psi|h psi> and |h psi|^2; uneven
    axes and twists, so that every axis has its own transform length and
    wavenumbers; 120 states at 24^3 take two chunks (about 108 states of psi
    and h psi per 48 MB)."""
    rng = np.random.default_rng(23 + I)
    with Ctx(grid, twist=twist, prec=B.SKY_F32, max_states=I) as c:
        g = c.grid
        psi = _r32(IN.random_spinors(g.n, I, rng))
        U, Bf, W = _fields(g, rng)
        want = O.apply_h(psi, U, Bf, W, g)
        e_w, n_w = O.sp_energies(psi, want, g)
        assert B.sky_tune_get(c.ctx, B.SKY_KNOB_FUSED_H) == (1 if max(grid) <= 24 else 0)
        out = {}
        for fused in (1, 0):
            B.sky_tune_set(c.ctx, B.SKY_KNOB_FUSED_H, fused)
            assert B.sky_tune_get(c.ctx, B.SKY_KNOB_FUSED_H) == fused
            d_h = torch.zeros(psi.shape, dtype=torch.complex64, device="cuda:0")
            eps = torch.zeros(I, dtype=torch.float64, device="cuda:0")
            hn2 = torch.zeros(I, dtype=torch.float64, device="cuda:0")
            B.sky_apply_h(c.ctx, dev(U), dev(Bf), dev(W), dev32(psi), d_h, I, eps, hn2)
            out[fused] = host(d_h)
            assert relerr(out[fused], want) < REL32, fused
            assert relerr(host(eps), e_w) < REL32, fused
            assert relerr(host(hn2), n_w) < REL32, fused
        assert relerr(out[1], out[0]) < REL32
    with Ctx((64, 48, 16), prec=B.SKY_F32, max_states=2) as c64:
        assert B.sky_tune_get(c64.ctx, B.SKY_KNOB_FUSED_H) == 0   # axes beyond 32: general path
        with pytest.raises(B.SkyError):
            B.sky_tune_set(c64.ctx, B.SKY_KNOB_FUSED_H, 1)


def test_fp32_overlap_and_rotate():
    rng = np.random.default_rng(22)
    with Ctx((32, 32, 32), prec=B.SKY_F32, max_states=70) as c:
        g = c.grid
        I = 67
        a, b = _r32(IN.random_spinors(g.n, I, rng)), _r32(IN.random_spinors(g.n, I, rng))
        X = torch.zeros((I, I), dtype=torch.complex128, device="cuda:0")
        B.sky_overlap(c.ctx, dev32(a), dev32(b), I, X)
        # 4-digit exact split products: digits to 2^-32 of each row's scale
        assert relerr(host(X), O.overlap(a, b, g)) < 1e-8
        M = rng.standard_normal((I, I)) + 1j * rng.standard_normal((I, I))
        out = torch.zeros(a.shape, dtype=torch.complex64, device="cuda:0")
        B.sky_rotate(c.ctx, dev32(a), dev(M), I, out)
        assert relerr(host(out), O.rotate(a, M)) < 1e-6


# ------------------------------------------------------------ split-BF16 forms
# Tensor-core contractions of FP32 spinors.  A 2-way bf16 split with 3 products
# keeps ~16 significant bits per product (error ~2^-17 of the summed |terms|);
# a 3-way split with 6 products keeps ~24 bits, which leaves the tensor cores'
# FP32 accumulation as the limit: a systematic bias of up to ~1e-5 of the
# largest entry over the ~1000-term runs of one K-split (measured 8.7e-6 at
# 24^3, I = 150).  Tolerances relative to the largest entry.
TC_TOL = {B.SKY_F32_BF16X3: 4e-5, B.SKY_F32_BF16X6: 2e-5}


@pytest.mark.parametrize("prec", [B.SKY_F32_BF16X3, B.SKY_F32_BF16X6])
@pytest.mark.parametrize("grid,I", [((16, 16, 16), 37), ((24, 24, 24), 150), ((12, 16, 20), 5)])
def test_tc_overlap_and_rotate(prec, grid, I):
    rng = np.random.default_rng(31 + I)
    with Ctx(grid, prec=prec, max_states=I) as c:
        g = c.grid
        a = _r32(O.orthonormalize(IN.random_superpositions(g.n, g.dx, I, rng), g))
        b = _r32(a + 0.05 * IN.random_spinors(g.n, I, rng) / np.sqrt(g.G))
        X = torch.zeros((I, I), dtype=torch.complex128, device="cuda:0")
        B.sky_overlap(c.ctx, dev32(a), dev32(b), I, X)
        B.sky_sync(c.ctx)
        assert relerr(host(X), O.overlap(a, b, g)) < TC_TOL[prec]
        B.sky_overlap(c.ctx, dev32(a), dev32(a), I, X)
        Xg = host(X)
        assert relerr(Xg, O.overlap(a, a, g)) < TC_TOL[prec]
        off = ~np.eye(I, dtype=bool)
        assert np.max(np.abs((Xg - Xg.conj().T)[off])) == 0.0   # mirrored lower triangle
        M = (rng.standard_normal((I, I)) + 1j * rng.standard_normal((I, I))) / np.sqrt(I)
        out = torch.zeros(a.shape, dtype=torch.complex64, device="cuda:0")
        B.sky_rotate(c.ctx, dev32(a), dev(M), I, out)
        assert relerr(host(out), O.rotate(a, M)) < TC_TOL[prec]


# Per-nucleon energy and level bounds of the FP32 forms over eight iterations
# of the 16^3 workload (E passes through zero there, so bounds are absolute).
FORM_TOL = {B.SKY_F32: (5e-6, 5e-4), B.SKY_F32_BF16X3: (5e-5, 5e-3), B.SKY_F32_BF16X6: (5e-6, 5e-4)}


@pytest.mark.parametrize("prec", [B.SKY_F32, B.SKY_F32_BF16X3, B.SKY_F32_BF16X6])
def test_fp32_forms_follow_the_fp64_iteration(prec):
    """Eight iterations of the 16^3, 16 n + 16 p workload in the FP32 forms stay
    within the stated distance of the FP64 oracle: |dE|/A (MeV) and the
    single-particle levels (MeV); also reports rho and orthonormality errors."""
    from paper_1610_07522_gb300.solver import Solver
    e_tol, lam_tol = FORM_TOL[prec]
    w = IN.WORKLOADS["sly4_16cubed_16n16p_fp64"]
    inp = IN.make_inputs(w)
    s = Solver(w, prec=prec)
    s.load(inp["psi0"])
    ora = _oracle_run(w, inp, 8)
    A = w.N + w.Z
    worst = {"dE/A": 0.0, "dlam": 0.0, "drho": 0.0}
    for k in range(8):
        s.step()
        E, de, _ = s.energy()
        lam = host(s.lam)
        dE = abs(E - ora[k]["E"]) / A
        dl = max(np.max(np.abs(np.sort(lam[:w.N]) - np.sort(ora[k]["lam"][0]))),
                 np.max(np.abs(np.sort(lam[w.N:]) - np.sort(ora[k]["lam"][1]))))
        dr = relerr(host(s.rho), ora[k]["rho"].reshape(2, -1))
        worst = {"dE/A": max(worst["dE/A"], dE), "dlam": max(worst["dlam"], dl),
                 "drho": max(worst["drho"], dr)}
        assert dE <= e_tol, (k, E, ora[k]["E"])
        assert dl <= lam_tol, k
    g = O.Grid(w.grid, w.dx)
    psi = [host(s.psi[q]).astype(np.complex128) for q in range(2)]
    ortho = max(np.max(np.abs(O.overlap(p, p, g) - np.eye(p.shape[0]))) for p in psi)
    print(f"form {prec}: max |dE|/A {worst['dE/A']:.2e} MeV, max |d eps| {worst['dlam']:.2e} MeV, "
          f"rho rel {worst['drho']:.2e}, ||Psi^H Psi - I||_max {ortho:.2e}")
    s.close()


def test_batched_loewdin_and_rayleigh_ritz():
    """Two species of different sizes in one batched solve: one overlap close to
    the identity (Newton-Schulz route), one far from it (eigendecomposition
    route); each matches the oracle's Loewdin factor and Ritz values."""
    rng = np.random.default_rng(41)
    with Ctx((16, 16, 16), max_states=40) as c:
        g = c.grid
        psi = O.orthonormalize(IN.random_superpositions(g.n, g.dx, 37, rng), g)
        near = psi + 1e-3 * IN.random_superpositions(g.n, g.dx, 37, rng) / np.sqrt(g.G)
        # S close to 4 I: outside the region (0, 3) where Newton-Schulz converges
        far = 2.0 * O.orthonormalize(IN.random_superpositions(g.n, g.dx, 16, rng), g)
        far = far + 0.05 * IN.random_superpositions(g.n, g.dx, 16, rng) / np.sqrt(g.G)
        Ss, Hs, Cw, Lw = [], [], [], []
        for phi in (near, far):
            U, Bf, W = _fields(g, rng)
            hphi = O.apply_h(phi, U, Bf, W, g)
            S, H = O.overlap(phi, phi, g), O.overlap(phi, hphi, g)
            Ss.append(S); Hs.append(H); Cw.append(O.loewdin(S)); Lw.append(O.rayleigh_ritz(S, H)[1])
        I = [37, 16]
        dS = [dev(x) for x in Ss]; dH = [dev(x) for x in Hs]
        C = [torch.zeros_like(x) for x in dS]; M = [torch.zeros_like(x) for x in dS]
        lam = [torch.zeros(n, dtype=torch.float64, device="cuda:0") for n in I]
        B.sky_stats(c.ctx, reset=True)
        B.sky_orthonormalize_batched(c.ctx, dS, I, C)
        B.sky_subspace_diag_batched(c.ctx, dH, C, I, M, lam)
        B.sky_sync(c.ctx)
        st = B.sky_stats(c.ctx)
        assert st["loewdin_calls"] == 2 and st["loewdin_newton_schulz"] == 1
        for b in range(2):
            assert relerr(host(C[b]), Cw[b]) < 1e-11
            assert np.max(np.abs(host(lam[b]) - Lw[b])) < 1e-9
            Mg = host(M[b])
            assert np.max(np.abs(Mg.conj().T @ Ss[b] @ Mg - np.eye(I[b]))) < 1e-11


@pytest.mark.parametrize("case", [CASES[2], CASES[3], CASES[4]])
def test_apply_h_and_densities_in_every_line_arithmetic(case):
    """The FP64 form's derivative passes as the digit-split operator on the
    tensor cores (the default, SKY_KNOB_LINE_ARITH = 2), as FFT line passes in
    double-float arithmetic (1) and in FP64 (0): all within the FP64 per-call
    tolerance of the oracle; FP32 contexts accept only 0."""
    rng = np.random.default_rng(77)
    with Ctx(*case) as c:
        g = c.grid
        I = 4
        psi = IN.random_spinors(g.n, I, rng)
        U, Bf, W = _fields(g, rng)
        want = O.apply_h(psi, U, Bf, W, g)
        rho_w, tau_w, J_w, dJ_w = O.densities(psi, g)
        assert B.sky_tune_get(c.ctx, B.SKY_KNOB_LINE_ARITH) == 2
        for arith in (2, 1, 0):
            B.sky_tune_set(c.ctx, B.SKY_KNOB_LINE_ARITH, arith)
            d_h = torch.zeros(psi.shape, dtype=torch.complex128, device="cuda:0")
            B.sky_apply_h(c.ctx, dev(U), dev(Bf), dev(W), dev(psi), d_h, I)
            assert relerr(host(d_h), want) < REL, arith
            rho = torch.zeros(g.G, dtype=torch.float64, device="cuda:0")
            tau, dJ = torch.zeros_like(rho), torch.zeros_like(rho)
            J = torch.zeros(3 * g.G, dtype=torch.float64, device="cuda:0")
            B.sky_densities(c.ctx, dev(psi), I, rho, tau, J, dJ)
            assert relerr(host(tau), tau_w.ravel()) < REL, arith
            assert relerr(host(J), J_w.ravel()) < REL, arith
    with Ctx((16, 16, 16), prec=B.SKY_F32) as c32:
        assert B.sky_tune_get(c32.ctx, B.SKY_KNOB_LINE_ARITH) == 0
        for bad in (1, 2):
            with pytest.raises(B.SkyError):
                B.sky_tune_set(c32.ctx, B.SKY_KNOB_LINE_ARITH, bad)


def test_tensor_core_derivative_many_tiles_ragged_and_in_place():
    """The operator kernel on 24^3 with 37 spinors (74 arrays: 42 624 lines per
    axis, 333 tiles of 128 with a ragged last tile; more tiles than SMs, so
    every CTA loops), through apply_h (gradient out of place, divergence in
    place) and against the FFT form in FP64 on the same context."""
    rng = np.random.default_rng(5)
    with Ctx((24, 24, 24), twist=(0.7, -0.3, 1.9)) as c:
        g = c.grid
        I = 37
        psi = IN.random_spinors(g.n, I, rng)
        U, Bf, W = _fields(g, rng)
        d_psi, dU, dB, dW = dev(psi), dev(U), dev(Bf), dev(W)
        out = {}
        for arith in (2, 0):
            B.sky_tune_set(c.ctx, B.SKY_KNOB_LINE_ARITH, arith)
            d_h = torch.zeros(psi.shape, dtype=torch.complex128, device="cuda:0")
            B.sky_apply_h(c.ctx, dU, dB, dW, d_psi, d_h, I)
            out[arith] = host(d_h)
        assert relerr(out[2], out[0]) < REL
        idx = [0, 17, 36]
        want = O.apply_h(psi[idx], U, Bf, W, g)
        assert relerr(out[2][idx], want) < REL


def test_apply_h_across_magnitudes():
    """Spinors scaled by 1e-28 ... 1e20 and one with exact zeros: the
    double-float passes convert doubles by their bit patterns inside
    2^-74 <= |x| < 2^127 and through FP64 conversions outside (zeros, smaller
    values); h is linear, so each spinor is compared with the oracle relative
    to its own largest value."""
    rng = np.random.default_rng(91)
    with Ctx((16, 16, 16), twist=(0.2, -0.4, 0.9)) as c:
        g = c.grid
        scales = [1e-28, 1e-21, 3e-9, 1.0, 7e5, 1e20]
        psi = IN.random_spinors(g.n, len(scales) + 1, rng)
        for a, s in enumerate(scales):
            psi[a] *= s
        psi[-1, 1] = 0.0                       # spin-down component identically zero
        psi[-1, 0, :, 3:9] = 0.0               # and a slab of zeros in spin-up
        U, Bf, W = _fields(g, rng)
        want = O.apply_h(psi, U, Bf, W, g)
        d_h = torch.zeros(psi.shape, dtype=torch.complex128, device="cuda:0")
        B.sky_apply_h(c.ctx, dev(U), dev(Bf), dev(W), dev(psi), d_h, psi.shape[0])
        got = host(d_h)
        for a in range(psi.shape[0]):
            assert relerr(got[a], want[a]) < REL, a


@pytest.mark.parametrize("case", [CASES[2], CASES[3], CASES[4]])
def test_damped_step_correction_in_every_arithmetic(case):
    """The damped step's correction psi - phi (the preconditioned residual,
    small beside psi) against the oracle's, with and without a per-voxel
    weight, in the three arithmetics of the FP64 form: the 3D transform pair
    as six DFT operator products on the tensor cores (default), FFT line
    passes in FP64 (0) -- (1) keeps the FFT passes as well."""
    rng = np.random.default_rng(17)
    with Ctx(*case) as c:
        g = c.grid
        I = 5
        psi = IN.random_spinors(g.n, I, rng)
        hpsi = IN.random_spinors(g.n, I, rng) * 30.0
        eps = rng.uniform(-40, 10, I)
        wv = (0.5 + rng.uniform(0.0, 1.5, g.shape)).astype(np.float32)
        base = O.damped_step(psi, hpsi, eps, g, P["hb2m_n"], 0.45, 100.0)
        for arith in (2, 1, 0):
            B.sky_tune_set(c.ctx, B.SKY_KNOB_LINE_ARITH, arith)
            for w in (None, wv):
                want = (psi - base) * (1.0 if w is None else w.astype(np.float64)[None, None])
                phi = torch.zeros(psi.shape, dtype=torch.complex128, device="cuda:0")
                B.sky_damped_step(c.ctx, 0, dev(psi), dev(hpsi), dev(eps), phi, I, 0.45, 100.0,
                                  None if w is None else dev(w))
                assert relerr(psi - host(phi), want) < REL, (arith, w is None)


@pytest.mark.parametrize("case", [CASES[1], CASES[3], CASES[4]])
def test_derivative_every_axis(case):
    """sky_derivative against the oracle's spectral derivative (twisted
    wavenumbers, Nyquist kept), every axis, out of place and in place, in the
    three arithmetics of the FP64 form; the FP32 form within its bound."""
    rng = np.random.default_rng(23)
    with Ctx(*case) as c:
        g = c.grid
        n = 7
        f = IN.random_spinors(g.n, n, rng).reshape((2 * n,) + g.shape)[:n]
        for arith in (2, 1, 0):
            B.sky_tune_set(c.ctx, B.SKY_KNOB_LINE_ARITH, arith)
            for ax in range(3):
                want = np.stack([O.deriv(f[k], ax, g) for k in range(n)])
                out = torch.zeros(f.shape, dtype=torch.complex128, device="cuda:0")
                B.sky_derivative(c.ctx, ax, dev(f), out, n)
                assert relerr(host(out), want) < REL, (arith, ax)
                inp = dev(f)
                B.sky_derivative(c.ctx, ax, inp, inp, n)
                assert relerr(host(inp), want) < REL, (arith, ax, "in place")
    with Ctx(case[0], case[1], case[2], prec=B.SKY_F32) as c32:
        g = c32.grid
        f = IN.random_spinors(g.n, 2, rng).reshape((4,) + g.shape)
        for ax in range(3):
            want = np.stack([O.deriv(f[k], ax, g) for k in range(4)])
            out = torch.zeros(f.shape, dtype=torch.complex64, device="cuda:0")
            B.sky_derivative(c32.ctx, ax, dev(f.astype(np.complex64)), out, 4)
            assert relerr(host(out), want) < 4e-6, ax
