"""Time-dependent stepping on the GPU against the FP64 oracle
(oracle/td_oracle.py): the Taylor propagator sky_td_taylor per call (random
smooth fields and states, twisted and ragged grids, orders 1-6; FP64 within
1e-12 of the largest magnitude, FP32 within 4e-6 like the other FP32 calls),
five self-consistent predictor-corrector steps of both species with Coulomb
(energies within 1e-10 relative, states within 1e-10), and over 40 steps of
the 16^3 workload: orthonormality kept to 1e-9 without any
orthonormalisation and the energy of the functional conserved."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from oracle import td_oracle as T
from paper_1610_07522_gb300 import binding as B
from paper_1610_07522_gb300 import inputs as IN
from paper_1610_07522_gb300.solver import Solver
from paper_1610_07522_gb300.td import HBARC, TimeStepper

pytestmark = pytest.mark.gpu

P = dict(IN.SLY4)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def relerr(got, want):
    return float(np.max(np.abs(got - want)) / np.max(np.abs(want)))


@pytest.mark.parametrize("prec", [B.SKY_F64, B.SKY_F32])
@pytest.mark.parametrize("grid,twist,order", [((16, 16, 16), (0.0, 0.0, 0.0), 6),
                                              ((12, 16, 20), (0.3, -1.2, 2.0), 4),
                                              ((8, 8, 8), (0.0, 0.5, 0.0), 1)])
def test_taylor_propagator_matches_oracle(prec, grid, twist, order):
    rng = np.random.default_rng(60 + order)
    g = O.Grid(grid, (1.0, 1.0, 1.0), twist)
    I = 5
    psi = IN.random_spinors(g.n, I, rng)
    if prec == B.SKY_F32:
        psi = psi.astype(np.complex64).astype(np.complex128)
    U = IN.random_smooth_field(g.n, rng, -40.0, 30.0)
    Bf = IN.random_smooth_field(g.n, rng, 20.0, 6.0)
    W = np.stack([IN.random_smooth_field(g.n, rng, 0.0, 10.0) for _ in range(3)])
    dt = 0.2
    want = T.taylor_step(psi, U, Bf, W, g, dt, order)
    ct = torch.complex128 if prec == B.SKY_F64 else torch.complex64
    c = B.sky_init(grid, (1.0, 1.0, 1.0), P, False, twist, prec, I,
                   torch.cuda.current_stream().cuda_stream)
    try:
        d_psi = dev(psi).to(ct)
        out = torch.zeros_like(d_psi)
        work = torch.zeros((2,) + tuple(d_psi.shape), dtype=ct, device="cuda:0")
        B.sky_td_taylor(c, dev(U), dev(Bf), dev(W), d_psi, out, work, I, dt / HBARC, order)
        B.sky_sync(c)
        got = out.cpu().numpy().astype(np.complex128)
        assert relerr(got, want) < (1e-12 if prec == B.SKY_F64 else 4e-6)
        with pytest.raises(B.SkyError):
            B.sky_td_taylor(c, dev(U), dev(Bf), dev(W), d_psi, d_psi, work, I, 0.1, order)
    finally:
        B.sky_destroy(c)


def _workload():
    return IN.Workload(name="td_8cubed", grid=(8, 8, 8), dx=(1.0, 1.0, 1.0), N=4, Z=3,
                       coulomb=True, twist=(0.3, -0.2, 0.5), seed=11)


@pytest.mark.parametrize("concurrent", [False, True])
def test_self_consistent_steps_match_oracle(concurrent):
    w = _workload()
    inp = IN.make_inputs(w)
    g = O.Grid(w.grid, w.dx, w.twist)
    st = O.initial_state(inp["psi0"], g, P, True)
    st.U, st.B, st.W = T.field_of(st.psi, g, P, True)[:3]
    s = Solver(w, prec=B.SKY_F64, concurrent_species=concurrent)
    try:
        s.load(inp["psi0"])
        ts = TimeStepper(s, order=6)
        ts.init_fields()
        for step in range(5):
            rec = T.td_step(st, g, P, True, 0.2)
            ts.step(0.2)
            E = ts.energy()
            assert abs(E - rec["E"]) <= 1e-10 * abs(rec["E"]), step
        for q in range(2):
            assert relerr(s.psi[q].cpu().numpy(), st.psi[q]) < 1e-10
    finally:
        s.close()


def test_long_run_keeps_orthonormality_and_energy():
    w = IN.WORKLOADS["sly4_16cubed_16n16p_fp64"]
    inp = IN.make_inputs(w)
    s = Solver(w, prec=B.SKY_F64)
    try:
        s.load(inp["psi0"])
        ts = TimeStepper(s, order=6)
        ts.init_fields()
        E0 = ts.energy()
        for _ in range(40):
            ts.step(0.1)
        E = ts.energy()
        S = torch.zeros((16, 16), dtype=torch.complex128, device="cuda:0")
        for q in range(2):
            B.sky_overlap(s.ctx, s.psi[q], s.psi[q], 16, S)
            B.sky_sync(s.ctx)
            assert np.max(np.abs(S.cpu().numpy() - np.eye(16))) < 1e-9
        assert abs(E - E0) < 1e-5 * abs(E0)
    finally:
        s.close()
