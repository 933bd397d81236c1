"""The constant damping weight (Solver.set_constant_weight, the uniform step
size a learned weight is compared with) against the oracle's damped step
with the same weight: phi = psi - c (psi - phi_plain), eight full iterations
of the 16^3, 16 n + 16 p workload, FP64 form."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_1610_07522_gb300 import binding as B
from paper_1610_07522_gb300 import inputs as IN
from paper_1610_07522_gb300.solver import Solver

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("c", [1.5, 0.75])
def test_constant_weight_against_the_oracle(c):
    w = IN.WORKLOADS["sly4_16cubed_16n16p_fp64"]
    inp = IN.make_inputs(w)
    g = O.Grid(w.grid, w.dx, w.twist)
    st = O.initial_state(inp["psi0"], g, w.params, w.coulomb, inp.get("rho0"), inp.get("tau0"))
    s = Solver(w, prec=B.SKY_F64)
    s.set_constant_weight(c)
    s.load(inp["psi0"], inp.get("rho0"), inp.get("tau0"))

    def damp(q, U, Bq, W):
        return np.full(g.shape, c)

    for it in range(8):
        s.step()
        E = s.energy()[0]
        r = O.iterate(st, g, w.params, w.coulomb, w.x0, w.E0, damping=damp)
        assert abs(E - r["E"]) <= 1e-10 * abs(r["E"]), (it, E, r["E"])
        lam = s.lam.cpu().numpy()
        assert np.max(np.abs(np.sort(lam[:w.N]) - np.sort(r["lam"][0]))) < 1e-9
    s.set_constant_weight(None)
    s.close()
