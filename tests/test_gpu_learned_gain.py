"""What the trained damping network gains over the plain damped step (GPU).

The network is trained on the GPU by the library's own forward, backward and
Adam kernels, on samples from a plain FP64 trajectory of the 16^3, 16n+16p
workload (one weighted step trained to reach where four plain steps go).
Then the plain step and the learned step each run to |dE/A| < 1e-6 MeV from
the same initial state.  The learned run must take clearly fewer iterations
and reach the same fixed point: the plain converged state is the reference.
The stopping rule |dE/A| < 1e-6 per iteration leaves each run short of the
exact fixed point by an amount that scales with its step size, so the two
final energies are compared at 1e-4 MeV per nucleon.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1610_07522_gb300 import binding as B
from paper_1610_07522_gb300 import inputs as IN
from paper_1610_07522_gb300 import learned
from paper_1610_07522_gb300.solver import Solver

pytestmark = pytest.mark.gpu

WL = "sly4_16cubed_16n16p_fp64"
SNAPS = [0, 2, 5, 12, 25, 60, 120, 180, 240, 360, 480, 600, 720, 840, 960]


def _run(w, net=None, maxit=3000):
    inp = IN.make_inputs(w)
    s = Solver(w, prec=B.SKY_F64)
    if net is not None:
        s.set_damping(net)
    s.load(inp["psi0"], inp.get("rho0"), inp.get("tau0"))
    hist, conv = s.run(maxit=maxit)
    lam = s.lam.cpu().numpy().copy()
    out = {"conv": conv, "its": len(hist), "E_A": hist[-1]["E"] / s.A, "lam": lam,
           "fallbacks": s.damping_fallbacks}
    s.close()
    return out


def test_trained_network_converges_faster_to_the_same_state():
    w = IN.WORKLOADS[WL]
    plain = _run(w)
    assert plain["conv"]
    inp = IN.make_inputs(w)
    s = Solver(w, prec=B.SKY_F64)
    s.load(inp["psi0"], inp.get("rho0"), inp.get("tau0"))
    samples = learned.collect(s, SNAPS, ahead=4)
    assert len(samples) == 2 * len(SNAPS)
    net = learned.DampingNet("cuda:0", seed=0)
    loss_plain = learned.sample_loss(net, samples, weight_one=True)
    learned.train(net, samples, 300, lr=3e-3)
    loss_trained = learned.sample_loss(net, samples)
    assert loss_trained < 0.5 * loss_plain
    lrn = _run(w, net)
    s.close()
    assert lrn["conv"]
    assert lrn["its"] < 0.8 * plain["its"], (lrn["its"], plain["its"])
    assert abs(lrn["E_A"] - plain["E_A"]) < 1e-4
    assert np.max(np.abs(lrn["lam"] - plain["lam"])) < 5e-3
