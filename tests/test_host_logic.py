"""Host logic of the iteration drivers (no GPU): the stop rule |E_n/A -
E_{n-1}/A| < tol held for `window` iterations, the escalation of the GEMM
form, the learned weight's fallback on an energy rise, and the batched
driver's per-box bookkeeping, each driven by a scripted energy sequence on a
stand-in object (the GPU calls replaced)."""
import types

import pytest

from paper_1610_07522_gb300.batched import BatchSolver
from paper_1610_07522_gb300.solver import Solver


def fake_solver(energies, A=10, damping=False):
    s = object.__new__(Solver)
    s.A = A
    s.w = types.SimpleNamespace(maxit=len(energies), tol=1e-6)
    s.damping_on = damping
    s.damping_scale = 1.0
    s.damping_fallbacks = 0
    s.rise_tol = 1e-5
    s.min_scale = 1.0 / 16.0
    s.graph = None
    s.precs = []
    seq = iter(energies)
    s.step = lambda frozen=False: None
    s.energy = lambda: (next(seq), 0.0, None)
    s.set_prec = lambda p: s.precs.append(p)
    return s


def test_stop_rule_plain_and_windowed():
    A = 10
    E = [-1.0, -2.0, -2.5, -2.5 - 5e-6, -2.5 - 6e-6, -2.5 - 6.5e-6, -2.5 - 6.7e-6, -3.0]
    hist, conv = fake_solver(E, A).run(window=1)
    assert conv and len(hist) == 4                 # first change below 1e-6 per nucleon
    hist, conv = fake_solver(E, A).run(window=3)
    assert conv and len(hist) == 6                 # three in a row
    # a single small change inside a large move does not end a windowed run
    E2 = [-1.0, -2.0, -2.0 - 1e-7, -3.0, -4.0]
    hist, conv = fake_solver(E2, A).run(window=2)
    assert not conv and len(hist) == 5


def test_escalation_then_stop():
    A = 1
    E = [0.0, -1.0, -1.0 - 1e-5, -1.0 - 2e-5, -1.0 - 2.1e-5, -1.0 - 2.1e-5 - 1e-7,
         -1.0 - 2.1e-5 - 2e-7, -1.0 - 2.1e-5 - 2.5e-7]
    s = fake_solver(E, A)
    hist, conv = s.run(tol=1e-6, window=2, escalate=(2e-5, 1))
    assert s.precs == [1]
    esc = next(h["it"] for h in hist if "escalated" in h)
    assert esc == 3                                 # two changes below 2e-5 (its 2nd and 3rd)
    assert conv and hist[-1]["it"] > esc            # the stop rule counts only after it


def test_learned_fallback_halves_then_turns_off():
    A = 1
    E = [0.0, -1.0, -0.5, -0.4, -0.3, -0.2, -0.1]   # every step a rise
    s = fake_solver(E, A, damping=True)
    hist, conv = s.run(tol=1e-9)
    assert not conv
    assert s.damping_fallbacks == 5
    assert s.damping_scale == 1.0 / 32.0 and not s.damping_on
    assert [h.get("fallback") for h in hist if "fallback" in h] == [0.5, 0.25, 0.125, 0.0625, 0.03125]


def test_callback_ends_the_run():
    s = fake_solver([0.0, -1.0, -2.0, -3.0], 1)
    hist, conv = s.run(callback=lambda it, rec: it == 1)
    assert not conv and len(hist) == 2


def test_batched_run_bookkeeping():
    b = object.__new__(BatchSolver)
    boxes = [types.SimpleNamespace(A=10, damping_on=False), types.SimpleNamespace(A=10, damping_on=True,
             rise_tol=1e-5, damping_scale=1.0, damping_fallbacks=0, min_scale=0.3)]
    b.boxes = boxes
    b.graph = object()
    b.graph_stale = False
    # box 0 converges after the window; box 1 rises twice (two fallbacks: 1/4 falls below
    # its minimum scale 0.3, so the plain step from then on) and converges later
    E0 = [-1.0, -2.0, -2.0, -2.0, -2.0, -2.0, -2.0, -2.0, -2.0, -2.0]
    E1 = [-1.0, -0.5, -0.4, -0.4, -0.4, -0.4, -0.4, -0.4, -0.4, -0.4]
    it = iter(range(len(E0)))
    cur = {}
    b.step = lambda: cur.__setitem__("k", next(it))
    b.energies = lambda check_status=True: [(E0[cur["k"]], 0.0), (E1[cur["k"]], 0.0)]
    done, E_done = b.run(maxit=len(E0), tol=1e-6, window=3)
    assert done == [5, 6]
    assert E_done[0] == pytest.approx(-0.2) and E_done[1] == pytest.approx(-0.04)
    assert boxes[1].damping_fallbacks == 2 and not boxes[1].damping_on
    assert b.graph_stale                              # a fallback changes the launch arguments
