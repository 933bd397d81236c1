"""Failure detection on the GPU without a GPU fault: every failure is made
on the host side (bad input data, a wait budget of zero, a sweep cap of
one), the device reports it in the status word, sky_sync raises it, and the
context stays usable for the next, correct call."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_1610_07522_gb300 import binding as B
from paper_1610_07522_gb300 import inputs as IN

pytestmark = pytest.mark.gpu

P = dict(IN.SLY4)


def _ctx(n=40):
    return B.sky_init((8, 8, 8), (1.0, 1.0, 1.0), P, True, (0.0, 0.0, 0.0), B.SKY_F64, n,
                      torch.cuda.current_stream().cuda_stream)


def _problem(rng, n):
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    S = 3.0 * np.eye(n) + (A @ A.conj().T) / n            # far from I: eigendecomposition route
    Hm = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return S, 5.0 * (Hm + Hm.conj().T)


def _solve(ctx, S, H):
    n = S.shape[0]
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    C = torch.zeros((n, n), dtype=torch.complex128, device="cuda:0")
    M = torch.zeros_like(C)
    lam = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    B.sky_orthonormalize(ctx, d(S), n, C)
    B.sky_subspace_diag(ctx, d(H), C, n, M, lam)
    return lam


def test_nan_density_sets_enan():
    c = _ctx()
    G = 512
    rho = torch.full((2, G), 0.01, dtype=torch.float64, device="cuda:0")
    rho[1, 17] = float("nan")
    tau = torch.zeros_like(rho)
    divJ = torch.zeros_like(rho)
    out = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    B.sky_energy(c, rho, tau, divJ, out)
    with pytest.raises(B.SkyError) as ei:
        B.sky_sync(c)
    assert ei.value.status == B.SKY_ENAN
    rho[1, 17] = 0.01
    B.sky_energy(c, rho, tau, divJ, out)
    B.sky_sync(c)                                # usable again
    B.sky_destroy(c)


def test_wait_budget_runs_out_with_etimeout_and_the_context_recovers():
    rng = np.random.default_rng(71)
    c = _ctx()
    S, H = _problem(rng, 40)
    default = B.sky_tune_get(c, B.SKY_KNOB_WAIT_SPINS)
    assert default > 0
    B.sky_tune_set(c, B.SKY_KNOB_WAIT_SPINS, 0)   # every grid-barrier wait gives up at once
    _solve(c, S, H)
    with pytest.raises(B.SkyError) as ei:
        B.sky_sync(c)
    assert ei.value.status == B.SKY_ETIMEOUT
    B.sky_tune_set(c, B.SKY_KNOB_WAIT_SPINS, default)
    lam = _solve(c, S, H)
    B.sky_sync(c)
    want = O.rayleigh_ritz(S, H)[1]
    assert np.max(np.abs(lam.cpu().numpy() - want)) < 1e-9 * np.max(np.abs(want))
    B.sky_destroy(c)


def test_sweep_cap_sets_enoconv_and_the_context_recovers():
    rng = np.random.default_rng(72)
    c = _ctx()
    S, H = _problem(rng, 40)
    B.sky_tune_set(c, B.SKY_KNOB_JACOBI_MAX_SWEEPS, 1)
    _solve(c, S, H)
    with pytest.raises(B.SkyError) as ei:
        B.sky_sync(c)
    assert ei.value.status == B.SKY_ENOCONV
    B.sky_tune_set(c, B.SKY_KNOB_JACOBI_MAX_SWEEPS, 60)
    lam = _solve(c, S, H)
    B.sky_sync(c)
    want = O.rayleigh_ritz(S, H)[1]
    assert np.max(np.abs(lam.cpu().numpy() - want)) < 1e-9 * np.max(np.abs(want))
    B.sky_destroy(c)
