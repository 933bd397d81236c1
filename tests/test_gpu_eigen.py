"""The two FP64 eigensolvers behind every diagonalisation (GPU): the parallel
cyclic Jacobi method and the tridiagonal route (Householder reduction to real
tridiagonal form, Sturm bisection, inverse iteration, back-transformation),
selected with SKY_KNOB_EIGEN_METHOD.  Each is driven through
sky_subspace_diag with C = I (so H' = H and M holds the eigenvectors) on
seeded Hermitian matrices with random, near-degenerate (pairs split by
1e-12..1e-3, as Kramers pairs are near convergence) and exactly degenerate
spectra, and compared with the oracle's Rayleigh-Ritz (Sec. 3.3.2):
eigenvalues, orthonormality, residuals and, where the eigenvalue is isolated,
the eigenvector itself up to its phase."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_1610_07522_gb300 import binding as B
from paper_1610_07522_gb300 import inputs as IN

pytestmark = pytest.mark.gpu

METHODS = {"jacobi": B.SKY_EIG_JACOBI, "tridiagonal": B.SKY_EIG_TRIDIAGONAL}


def _ctx(nmax):
    return B.sky_init((8, 8, 8), (1.0, 1.0, 1.0), dict(IN.SLY4), True, (0.0, 0.0, 0.0),
                      B.SKY_F64, nmax, torch.cuda.current_stream().cuda_stream)


def _unitary(rng, n):
    q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    return q


def _matrix(kind, n, rng):
    if kind == "random":
        a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        return 10.0 * (a + a.conj().T)
    U = _unitary(rng, n)
    c = np.sort(rng.uniform(-60.0, 40.0, (n + 1) // 2))
    if kind == "pairs":
        sp = 10.0 ** rng.uniform(-12.0, -3.0, c.size)
        ev = np.concatenate([c - sp / 2, c + sp / 2])[:n]
    else:   # exactly degenerate: pairs and a 4-fold level
        ev = np.repeat(c, 2)[:n]
        ev[: min(4, n)] = c[0]
    H = (U * ev) @ U.conj().T
    return 0.5 * (H + H.conj().T)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _solve(ctx, H):
    n = H.shape[0]
    C = _dev(np.eye(n, dtype=np.complex128))
    M = torch.zeros((n, n), dtype=torch.complex128, device="cuda:0")
    lam = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    B.sky_subspace_diag(ctx, _dev(H), C, n, M, lam)
    B.sky_sync(ctx)
    return M.cpu().numpy(), lam.cpu().numpy()


def _check(H, M, lam, label):
    n = H.shape[0]
    Mw, lw = O.rayleigh_ritz(np.eye(n, dtype=np.complex128), H)
    nrm = max(1.0, float(np.max(np.abs(lw))))
    de = float(np.max(np.abs(lam - lw)))
    orth = float(np.max(np.abs(M.conj().T @ M - np.eye(n))))
    res = float(np.max(np.abs(H @ M - M * lam)))
    print(f"{label}: |d lambda| {de:.1e}, ||M^H M - I|| {orth:.1e}, residual {res:.1e} (||H|| {nrm:.0f})")
    assert de < 1e-12 * nrm * max(1, n // 100)
    assert orth < 1e-12
    assert res < 1e-12 * nrm
    gaps = np.minimum(np.diff(lw, prepend=-np.inf), np.diff(lw, append=np.inf))
    for j in np.flatnonzero(gaps > 1e-6 * nrm):
        k = int(np.argmax(np.abs(Mw[:, j])))
        ph = M[k, j] / Mw[k, j]
        assert abs(abs(ph) - 1.0) < 1e-8
        assert np.max(np.abs(M[:, j] - ph * Mw[:, j])) < 1e-8


@pytest.mark.parametrize("method", list(METHODS))
@pytest.mark.parametrize("kind", ["random", "pairs", "degenerate"])
@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 130, 300])
def test_eigensolver_against_oracle(method, kind, n):
    rng = np.random.default_rng(1000 * n + len(kind))
    H = _matrix(kind, n, rng)
    c = _ctx(max(n, 2))
    B.sky_tune_set(c, B.SKY_KNOB_EIGEN_METHOD, METHODS[method])
    B.sky_stats(c, reset=True)
    M, lam = _solve(c, H)
    st = B.sky_stats(c)
    B.sky_destroy(c)
    if method == "tridiagonal":
        assert st["tridiagonal_solves"] == 1 and st["jacobi_solves"] == 0
    else:
        assert st["jacobi_solves"] == 1 and st["tridiagonal_solves"] == 0
    _check(H, M, lam, f"{method} {kind} n={n}")


def test_auto_method_picks_the_tridiagonal_route_for_large_problems():
    rng = np.random.default_rng(5)
    c = _ctx(96)
    assert B.sky_tune_get(c, B.SKY_KNOB_EIGEN_METHOD) == B.SKY_EIG_AUTO
    B.sky_stats(c, reset=True)
    _solve(c, _matrix("random", 40, rng))
    _solve(c, _matrix("random", 96, rng))
    st = B.sky_stats(c)
    B.sky_destroy(c)
    assert st["jacobi_solves"] == 1 and st["tridiagonal_solves"] == 1


def test_batched_tridiagonal_route_uneven_sizes():
    """Two problems of different sizes (the neutron / proton pair of one box)
    in one batched launch sequence, each against the oracle."""
    rng = np.random.default_rng(9)
    sizes = [300, 130]
    Hs = [_matrix("pairs", sizes[0], rng), _matrix("random", sizes[1], rng)]
    c = _ctx(300)
    B.sky_tune_set(c, B.SKY_KNOB_EIGEN_METHOD, B.SKY_EIG_TRIDIAGONAL)
    dH = [_dev(h) for h in Hs]
    dC = [_dev(np.eye(n, dtype=np.complex128)) for n in sizes]
    M = [torch.zeros((n, n), dtype=torch.complex128, device="cuda:0") for n in sizes]
    lam = [torch.zeros(n, dtype=torch.float64, device="cuda:0") for n in sizes]
    B.sky_subspace_diag_batched(c, dH, dC, sizes, M, lam)
    B.sky_sync(c)
    B.sky_destroy(c)
    for b in range(2):
        _check(Hs[b], M[b].cpu().numpy(), lam[b].cpu().numpy(), f"batched b={b} n={sizes[b]}")


def test_batched_tridiagonal_teams_many_uneven_problems():
    """Forty problems of the sizes of the twist-averaged batch (both species of
    16^3, 20^3 and 24^3 boxes, plus a few others) in one batched solve: more
    than eight problems, so the reduction's blocks split into teams (several
    blocks for a large problem, small ones sharing a block); the automatic
    method must take the tridiagonal route, and every problem agrees with the
    oracle."""
    rng = np.random.default_rng(19)
    sizes = [290, 125, 168, 72, 86, 37] * 6 + [300, 17, 64, 3]
    kinds = ["random", "pairs", "degenerate"]
    Hs = [_matrix(kinds[b % 3], n, rng) for b, n in enumerate(sizes)]
    c = _ctx(300)
    B.sky_reserve_batch(c, len(sizes))
    B.sky_stats(c, reset=True)
    dH = [_dev(h) for h in Hs]
    dC = [_dev(np.eye(n, dtype=np.complex128)) for n in sizes]
    M = [torch.zeros((n, n), dtype=torch.complex128, device="cuda:0") for n in sizes]
    lam = [torch.zeros(n, dtype=torch.float64, device="cuda:0") for n in sizes]
    B.sky_subspace_diag_batched(c, dH, dC, sizes, M, lam)
    B.sky_sync(c)
    st = B.sky_stats(c)
    B.sky_destroy(c)
    assert st["tridiagonal_solves"] == len(sizes) and st["jacobi_solves"] == 0
    for b, n in enumerate(sizes):
        _check(Hs[b], M[b].cpu().numpy(), lam[b].cpu().numpy(),
               f"teams b={b} {kinds[b % 3]} n={n}")


def test_gated_loewdin_many_problems_by_teams():
    """Twelve overlaps, every third far from the identity: Newton-Schulz for
    the others, the eigendecomposition route (gated on the device) for those,
    all in one batched call whose tridiagonal launch runs only the gated
    problems' teams; every factor against the oracle's S^{-1/2}."""
    rng = np.random.default_rng(23)
    sizes = [150, 90, 64, 120, 70, 100, 66, 130, 80, 96, 110, 75]
    S = []
    for b, n in enumerate(sizes):
        if b % 3 == 0:
            X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
            S.append(X @ X.conj().T / n + 0.05 * np.eye(n))
        else:
            E = 1e-3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
            S.append(np.eye(n) + 0.5 * (E + E.conj().T))
    c = _ctx(150)
    B.sky_reserve_batch(c, len(sizes))
    B.sky_stats(c, reset=True)
    dS = [_dev(s_) for s_ in S]
    C = [torch.zeros((n, n), dtype=torch.complex128, device="cuda:0") for n in sizes]
    B.sky_orthonormalize_batched(c, dS, sizes, C)
    B.sky_sync(c)
    st = B.sky_stats(c)
    B.sky_destroy(c)
    assert st["tridiagonal_solves"] == 4 and st["jacobi_solves"] == 0
    for b in range(len(sizes)):
        Cw = O.loewdin(S[b])
        Cg = C[b].cpu().numpy()
        assert np.max(np.abs(Cg - Cw)) < 1e-10 * np.max(np.abs(Cw)), b


@pytest.mark.parametrize("n", [290, 125])
def test_split_bf16_context_products_with_padded_digit_rows(n):
    """A split-BF16 context sizes its digit buffers for the I x I products
    alone; with 2n not a multiple of 8 (290, 125) the digit rows are padded to
    the next multiple of 8, and the buffers must hold the padded rows (they
    once held 2n per row, and the last rows ran past the end).  Loewdin
    factor (Newton-Schulz with tensor-core products from 192 states) and
    Rayleigh-Ritz (tensor-core products from 96) against the oracle."""
    rng = np.random.default_rng(40 + n)
    c = B.sky_init((8, 8, 8), (1.0, 1.0, 1.0), dict(IN.SLY4), False, (0.0, 0.0, 0.0),
                   B.SKY_F32_BF16X3, 290, torch.cuda.current_stream().cuda_stream)
    E = 2e-3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    S = np.eye(n) + 0.5 * (E + E.conj().T)
    H = _matrix("random", n, rng)
    C = torch.zeros((n, n), dtype=torch.complex128, device="cuda:0")
    M = torch.zeros_like(C)
    lam = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    for _ in range(2):
        B.sky_orthonormalize(c, _dev(S), n, C)
        B.sky_subspace_diag(c, _dev(H), C, n, M, lam)
    B.sky_sync(c)
    B.sky_destroy(c)
    Cw = O.loewdin(S)
    assert np.max(np.abs(C.cpu().numpy() - Cw)) < 1e-11 * np.max(np.abs(Cw))
    _, want = O.rayleigh_ritz(S, H)
    assert np.max(np.abs(lam.cpu().numpy() - want)) < 1e-9 * max(1.0, np.max(np.abs(want)))
    Mg = M.cpu().numpy()
    assert np.max(np.abs(Mg.conj().T @ S @ Mg - np.eye(n))) < 1e-11


def test_loewdin_eigen_route_by_tridiagonal_solver():
    """An overlap far from the identity (S^{-1/2} from the eigendecomposition,
    Eq. Loewedin) at a size the tridiagonal route serves."""
    rng = np.random.default_rng(13)
    n = 150
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    S = 3.0 * np.eye(n) + (a @ a.conj().T) / n
    c = _ctx(n)
    B.sky_stats(c, reset=True)
    C = torch.zeros((n, n), dtype=torch.complex128, device="cuda:0")
    B.sky_orthonormalize(c, _dev(S), n, C)
    B.sky_sync(c)
    st = B.sky_stats(c)
    B.sky_destroy(c)
    Cg = C.cpu().numpy()
    assert st["loewdin_newton_schulz"] == 0 and st["tridiagonal_solves"] == 1
    Cw = O.loewdin(S)
    assert np.max(np.abs(Cg - Cw)) / np.max(np.abs(Cw)) < 1e-11
    assert np.max(np.abs(Cg.conj().T @ S @ Cg - np.eye(n))) < 1e-11


def test_tridiagonal_wait_budget_runs_out_with_etimeout_and_recovers():
    rng = np.random.default_rng(17)
    H = _matrix("random", 96, rng)
    c = _ctx(96)
    B.sky_tune_set(c, B.SKY_KNOB_EIGEN_METHOD, B.SKY_EIG_TRIDIAGONAL)
    default = B.sky_tune_get(c, B.SKY_KNOB_WAIT_SPINS)
    B.sky_tune_set(c, B.SKY_KNOB_WAIT_SPINS, 0)
    with pytest.raises(B.SkyError) as ei:
        _solve(c, H)
    assert ei.value.status == B.SKY_ETIMEOUT
    B.sky_tune_set(c, B.SKY_KNOB_WAIT_SPINS, default)
    M, lam = _solve(c, H)
    B.sky_destroy(c)
    _check(H, M, lam, "tridiagonal after a timeout")


def test_tridiagonal_route_beyond_shared_memory():
    """3700 states: the reduction's three work vectors per block no longer fit
    in shared memory and live in a per-block global buffer; the route must
    still be taken (no Jacobi fallback) and agree with the oracle."""
    n = 3700
    rng = np.random.default_rng(37)
    H = _matrix("random", n, rng)
    c = _ctx(n)
    B.sky_tune_set(c, B.SKY_KNOB_EIGEN_METHOD, B.SKY_EIG_TRIDIAGONAL)
    B.sky_stats(c, reset=True)
    M, lam = _solve(c, H)
    st = B.sky_stats(c)
    B.sky_destroy(c)
    assert st["tridiagonal_solves"] == 1 and st["jacobi_solves"] == 0
    _check(H, M, lam, f"tridiagonal random n={n}")


def test_gated_loewdin_batch_too_large_for_one_shared_memory_stays_tridiagonal():
    """Two 2000-state overlaps far from the identity (the eigendecomposition
    route, gated on the device): their work vectors together exceed shared
    memory, and a gated batch cannot be split into launch groups, so the
    larger problems' vectors move to the global buffer and the batch stays on
    the tridiagonal route (no Jacobi fallback)."""
    n = 2000
    rng = np.random.default_rng(41)
    S = []
    for _ in range(2):
        X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        S.append(X @ X.conj().T / n + 0.05 * np.eye(n))
    c = _ctx(n)
    B.sky_stats(c, reset=True)
    dS = [_dev(s_) for s_ in S]
    C = [torch.zeros((n, n), dtype=torch.complex128, device="cuda:0") for _ in range(2)]
    B.sky_orthonormalize_batched(c, dS, [n, n], C)
    B.sky_sync(c)
    st = B.sky_stats(c)
    B.sky_destroy(c)
    assert st["tridiagonal_solves"] == 2 and st["jacobi_solves"] == 0
    for b in range(2):
        Cw = O.loewdin(S[b])
        Cg = C[b].cpu().numpy()
        assert np.max(np.abs(Cg - Cw)) < 1e-10 * np.max(np.abs(Cw))
