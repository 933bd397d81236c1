"""The learned-weight form at the 64^3 scale of the 5600 n + 2400 p workload,
with a state count the oracle finishes in minutes (12 n + 6 p, Coulomb, blob
start): one iteration of the FP32 form with the plain step and one with a
fixed random network, each against one iteration of the FP64 oracle on the
same seeded inputs.  Bounds: the FP32 form's stated bounds of the 32^3
precision test (|dE|/A 5e-6 MeV, levels 5e-4 MeV, rho 1e-5 relative); the
FP32 network against the FP64 one adds ~1e-7 relative (the weight enters the
update linearly)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from oracle import precond_oracle as PO
from paper_1610_07522_gb300 import binding as B
from paper_1610_07522_gb300 import inputs as IN
from paper_1610_07522_gb300.solver import Solver

pytestmark = pytest.mark.gpu

W64 = IN.Workload(name="learned_64cubed_12n6p", grid=(64, 64, 64), dx=(1.0, 1.0, 1.0),
                  N=12, Z=6, coulomb=True, init="blobs", seed=4321)


def _theta():
    from paper_1610_07522_gb300 import learned
    rng = np.random.default_rng(21)
    theta = learned.init_params(3)
    parts = PO.unpack(theta.astype(np.float64).copy())
    parts["W3"][:] = 0.2 * rng.standard_normal(parts["W3"].shape)
    return PO.pack(parts).astype(np.float32)


@pytest.mark.parametrize("learned_weight", [False, True])
def test_one_iteration_at_64cubed(learned_weight):
    from paper_1610_07522_gb300 import learned
    w = W64
    inp = IN.make_inputs(w)
    g = O.Grid(w.grid, w.dx, w.twist)
    hb2m = (w.params["hb2m_n"], w.params["hb2m_p"])
    theta = _theta()
    damping = None
    if learned_weight:
        damping = lambda q, U, Bq, Wq: PO.forward(theta.astype(np.float64),
                                                  PO.features(U, Bq, Wq, hb2m[q]))[0]
    st = O.initial_state(inp["psi0"], g, w.params, w.coulomb, inp["rho0"], inp["tau0"])
    rec = O.iterate(st, g, w.params, w.coulomb, w.x0, w.E0, damping=damping)
    s = Solver(w, prec=B.SKY_F32)
    try:
        if learned_weight:
            s.set_damping(learned.DampingNet("cuda:0", theta=theta))
        s.load(inp["psi0"], inp["rho0"], inp["tau0"])
        s.step()
        E, _, _ = s.energy()
        A = w.N + w.Z
        assert abs(E - rec["E"]) / A < 5e-6
        lam = s.lam.cpu().numpy()
        dl = max(np.max(np.abs(np.sort(lam[:w.N]) - np.sort(rec["lam"][0]))),
                 np.max(np.abs(np.sort(lam[w.N:]) - np.sort(rec["lam"][1]))))
        assert dl < 5e-4
        rho = s.rho.cpu().numpy()
        want = rec["rho"].reshape(2, -1)
        assert np.max(np.abs(rho - want)) / np.max(np.abs(want)) < 1e-5
    finally:
        s.close()
