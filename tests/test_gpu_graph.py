"""One iteration captured as a CUDA graph (Solver.capture) and replayed gives
the same states and energies, bit for bit, as the iterations enqueued call by
call: the same kernels on the same buffers, FP64 form, both species on their
own contexts and streams (the configuration bench.py times)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1610_07522_gb300 import binding as B
from paper_1610_07522_gb300 import inputs as IN
from paper_1610_07522_gb300.solver import Solver

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["sly4_16cubed_16n16p_fp64"])
def test_graph_replay_is_bit_identical(name):
    w = IN.WORKLOADS[name]
    inp = IN.make_inputs(w)
    runs = []
    for graph in (False, True):
        s = Solver(w, prec=B.SKY_F64, concurrent_species=True)
        s.load(inp["psi0"], inp.get("rho0"), inp.get("tau0"))
        s.step()                      # first-use work happens eagerly
        if graph:
            s.capture()
            assert s.launches_per_step > 50
        E = []
        for _ in range(6):
            s.step()
            E.append(s.energy()[0])
        s.sync()
        runs.append((E, [p.cpu().numpy() for p in s.psi], s.lam.cpu().numpy()))
        s.close()
    (Ea, pa, la), (Eb, pb, lb) = runs
    assert Ea == Eb
    for x, y in zip(pa, pb):
        assert np.array_equal(x, y)
    assert np.array_equal(la, lb)
