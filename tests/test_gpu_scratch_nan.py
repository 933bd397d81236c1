"""No kernel reads context scratch it has not written: with every buffer a
context allocates filled with NaN bytes (SKY_FILL_SCRATCH_NAN=1), iterations
of every precision form give the same results bit for bit as with ordinary
allocations.  (A read of an unwritten entry, even one multiplied by zero,
turns into NaN.)  Covers the FFT passes, the GEMMs of every form, both FP64
eigensolvers at odd and even sizes, densities, mean field and energy."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1610_07522_gb300 import binding as B
from paper_1610_07522_gb300 import inputs as IN
from paper_1610_07522_gb300.solver import Solver

pytestmark = pytest.mark.gpu


def _run(w, prec, eig, iters):
    inp = IN.make_inputs(w)
    s = Solver(w, prec=prec)
    s.set_eigen_method(eig)
    s.load(inp["psi0"], inp.get("rho0"), inp.get("tau0"))
    for _ in range(iters):
        s.step()
    E, de, _ = s.energy()
    out = (E, de, s.lam.cpu().numpy(), [p.cpu().numpy() for p in s.psi])
    s.close()
    return out


@pytest.mark.parametrize("prec", [B.SKY_F64, B.SKY_F32, B.SKY_F32_BF16X3, B.SKY_F32_BF16X6])
@pytest.mark.parametrize("eig", [B.SKY_EIG_TRIDIAGONAL, B.SKY_EIG_JACOBI])
def test_nan_filled_scratch_changes_nothing(monkeypatch, prec, eig):
    w = IN.Workload(name="scratch_nan", grid=(12, 16, 20), dx=(1.0, 1.0, 1.0), N=67, Z=33,
                    coulomb=True, twist=(0.3, -0.5, 0.2), init="blobs", seed=4242)
    monkeypatch.delenv("SKY_FILL_SCRATCH_NAN", raising=False)
    ref = _run(w, prec, eig, 3)
    monkeypatch.setenv("SKY_FILL_SCRATCH_NAN", "1")
    got = _run(w, prec, eig, 3)
    assert np.isfinite(got[0]) and got[0] == ref[0] and got[1] == ref[1]
    assert np.array_equal(got[2], ref[2])
    for a, b in zip(got[3], ref[3]):
        assert np.array_equal(a, b)
