"""Switching the GEMM form of a running FP32-spinor context (GPU):
sky_set_prec gives the same results as a context created in the target form,
and a split-BF16 run escalated to FP32 GEMMs near convergence reaches the
FP64 fixed point, which the split-BF16 form alone cannot (its orthonormality
error, about 1e-5, shifts E/A by more than the stop rule)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_1610_07522_gb300 import binding as B
from paper_1610_07522_gb300 import inputs as IN
from paper_1610_07522_gb300.solver import Solver

pytestmark = pytest.mark.gpu

P = dict(IN.SLY4)


def _ctx(prec, grid=(12, 16, 20)):
    return B.sky_init(grid, (1.0, 1.0, 1.0), P, False, (0.0, 0.0, 0.0), prec, 80,
                      torch.cuda.current_stream().cuda_stream)


def test_set_prec_matches_a_context_made_in_that_form():
    rng = np.random.default_rng(91)
    g = O.Grid((12, 16, 20), (1.0, 1.0, 1.0))
    I = 70
    a = torch.from_numpy(IN.random_spinors(g.n, I, rng).astype(np.complex64)).cuda()
    b = torch.from_numpy(IN.random_spinors(g.n, I, rng).astype(np.complex64)).cuda()
    c64 = _ctx(B.SKY_F64)
    with pytest.raises(B.SkyError):
        B.sky_set_prec(c64, B.SKY_F32)
    B.sky_destroy(c64)
    sw = _ctx(B.SKY_F32)
    out = {}
    for prec in (B.SKY_F32_BF16X3, B.SKY_F32_BF16X6, B.SKY_F32):
        B.sky_set_prec(sw, prec)
        ref = _ctx(prec)
        X1 = torch.zeros((I, I), dtype=torch.complex128, device="cuda:0")
        X2 = torch.zeros_like(X1)
        B.sky_overlap(sw, a, b, I, X1)
        B.sky_overlap(ref, a, b, I, X2)
        r1, r2 = torch.zeros_like(a), torch.zeros_like(a)
        B.sky_rotate(sw, a, X1, I, r1)
        B.sky_rotate(ref, a, X1, I, r2)
        torch.cuda.synchronize()
        assert torch.equal(X1, X2) and torch.equal(r1, r2), prec
        out[prec] = X1.cpu().numpy()
        B.sky_destroy(ref)
    B.sky_destroy(sw)
    want = O.overlap(a.cpu().numpy().astype(np.complex128), b.cpu().numpy().astype(np.complex128), g)
    # full products in the split forms vs the lower-triangle mirror of the oracle
    err = {p: np.max(np.abs(np.tril(out[p]) - np.tril(want))) / np.max(np.abs(want)) for p in out}
    # SKY_F32: 4-digit exact split products, digits to 2^-32 of each row's scale
    assert err[B.SKY_F32] < 1e-8 and err[B.SKY_F32_BF16X6] < 2e-5 and err[B.SKY_F32_BF16X3] < 4e-5


def test_escalated_split_bf16_run_reaches_the_fp64_fixed_point():
    w = IN.WORKLOADS["sly4_16cubed_16n16p_fp64"]
    inp = IN.make_inputs(w)
    res = {}
    for name, prec, esc in (("fp64", B.SKY_F64, None), ("x3_to_f32", B.SKY_F32_BF16X3, (2e-5, B.SKY_F32))):
        s = Solver(w, prec=prec)
        s.load(inp["psi0"])
        hist, conv = s.run(maxit=4000, window=5, escalate=esc)
        res[name] = (conv, hist[-1]["E"] / s.A, any("escalated" in h for h in hist))
        s.close()
    assert res["fp64"][0] and res["x3_to_f32"][0]
    assert res["x3_to_f32"][2]
    assert abs(res["x3_to_f32"][1] - res["fp64"][1]) < 1e-4


@pytest.mark.parametrize("prec", [B.SKY_F64, B.SKY_F32_BF16X3])
def test_concurrent_species_streams_give_the_same_iteration(prec):
    """Neutrons and protons on separate contexts and streams (joined for the
    batched eigensolve and the mean field): bit-identical to one stream."""
    w = IN.WORKLOADS["sly4_24cubed_280n120p_coulomb_fp64"]
    inp = IN.make_inputs(w)
    a = Solver(w, prec=prec)
    b = Solver(w, prec=prec, concurrent_species=True)
    assert b.concurrent and not a.concurrent
    for s in (a, b):
        s.load(inp["psi0"], inp["rho0"], inp["tau0"])
    for _ in range(3):
        a.step()
        b.step()
    Ea, Eb = a.energy(), b.energy()
    assert Ea[0] == Eb[0] and Ea[1] == Eb[1]
    assert torch.equal(a.psi[1], b.psi[1]) and torch.equal(a.rho, b.rho)
    a.close()
    b.close()


@pytest.mark.parametrize("prec", [B.SKY_F64, B.SKY_F32])
def test_split_eigensolve_chains_match_the_batched_solve(prec):
    """Each species' Loewdin and Rayleigh-Ritz solve on its own context and
    stream (two independent chains up to the densities) against the batched
    solve of both: the same iteration up to the order of the eigensolver's
    partial sums (its grid depends on the problems launched together)."""
    w = IN.WORKLOADS["sly4_24cubed_280n120p_coulomb_fp64"]
    inp = IN.make_inputs(w)
    a = Solver(w, prec=prec, concurrent_species=True)
    b = Solver(w, prec=prec, concurrent_species=True, split_eigensolve=True)
    assert b.split_eig and not a.split_eig
    for s in (a, b):
        s.load(inp["psi0"], inp["rho0"], inp["tau0"])
    for _ in range(3):
        a.step()
        b.step()
    Ea, Eb = a.energy(), b.energy()
    tol = 1e-11 if prec == B.SKY_F64 else 1e-6
    assert abs(Ea[0] - Eb[0]) <= tol * abs(Ea[0])
    la, lb = a.lam.cpu().numpy(), b.lam.cpu().numpy()
    assert np.max(np.abs(la - lb)) < (1e-9 if prec == B.SKY_F64 else 1e-3)
    a.close()
    b.close()
