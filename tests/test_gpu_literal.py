"""The paper's combined form of steps 3b-3e (Sec. 3.3.3) as a selectable
variant (GPU): per call against the oracle's combined_literal, and three
iterations of a twisted box (no Kramers degeneracy, so Z is unique up to
phases) against the oracle iteration with variant='paper_literal'."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_1610_07522_gb300 import binding as B
from paper_1610_07522_gb300 import inputs as IN
from paper_1610_07522_gb300.solver import Solver

pytestmark = pytest.mark.gpu

P = dict(IN.SLY4)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def test_literal_call_matches_oracle():
    rng = np.random.default_rng(51)
    ctx = B.sky_init((8, 8, 8), (1.0, 1.0, 1.0), P, False, (0.0, 0.0, 0.0), B.SKY_F64, 50,
                     torch.cuda.current_stream().cuda_stream)
    sizes = [50, 17]
    Ss, Hs = [], []
    for n in sizes:
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        S = np.eye(n) + 0.01 * (A + A.conj().T)
        Hm = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        Ss.append(S)
        Hs.append(5.0 * (Hm + Hm.conj().T) + np.diag(np.arange(n) * 2.0))
    C = [torch.zeros((n, n), dtype=torch.complex128, device="cuda:0") for n in sizes]
    M = [torch.zeros_like(x) for x in C]
    lam = [torch.zeros(n, dtype=torch.float64, device="cuda:0") for n in sizes]
    B.sky_orthonormalize_batched(ctx, [dev(x) for x in Ss], sizes, C)
    B.sky_subspace_diag_literal_batched(ctx, [dev(x) for x in Hs], C, sizes, M, lam)
    B.sky_sync(ctx)
    for b, n in enumerate(sizes):
        Mw, lw = O.combined_literal(Ss[b], Hs[b])
        assert np.max(np.abs(lam[b].cpu().numpy() - lw)) < 1e-9 * np.max(np.abs(lw))
        # distinct eigenvalues and the same phase convention: M is unique
        Mg = M[b].cpu().numpy()
        assert np.max(np.abs(Mg - Mw)) < 1e-10 * np.max(np.abs(Mw))
    B.sky_destroy(ctx)


def test_literal_iterations_match_oracle():
    w = IN.Workload(name="t", grid=(12, 16, 8), dx=(1.0, 0.9, 1.2), N=9, Z=7, coulomb=True,
                    twist=(1.0, -0.5, 2.2), init="blobs", seed=33)
    inp = IN.make_inputs(w)
    g = O.Grid(w.grid, w.dx, w.twist)
    st = O.initial_state(inp["psi0"], g, w.params, w.coulomb, inp["rho0"], inp["tau0"])
    s = Solver(w, prec=B.SKY_F64, variant="paper_literal")
    s.load(inp["psi0"], inp["rho0"], inp["tau0"])
    ex = Solver(w, prec=B.SKY_F64)
    ex.load(inp["psi0"], inp["rho0"], inp["tau0"])
    for k in range(3):
        rec = O.iterate(st, g, w.params, w.coulomb, w.x0, w.E0, variant="paper_literal")
        s.step()
        ex.step()
        E, _, _ = s.energy()
        assert abs(E - rec["E"]) <= 1e-10 * abs(rec["E"]), k
        lam = s.lam.cpu().numpy()
        assert np.max(np.abs(lam[:w.N] - rec["lam"][0])) < 1e-9
        assert np.max(np.abs(lam[w.N:] - rec["lam"][1])) < 1e-9
        rho = s.rho.cpu().numpy()
        assert np.max(np.abs(rho - rec["rho"].reshape(2, -1))) < 1e-10 * np.max(np.abs(rec["rho"]))
    # the variant really differs from the exact form during the iteration
    assert abs(ex.energy()[0] - s.energy()[0]) > 1e-9
    s.close()
    ex.close()
