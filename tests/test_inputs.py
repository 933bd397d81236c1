"""The seeded synthetic inputs shared by the oracle and the GPU path (CPU):
the workloads' sizes, the batched boxes' particle numbers (0.03 fm^-3,
proton fraction 0.3) and twists, the plane-wave shells of the trial states,
and the normalisation and shape of the blob and pasta starting densities."""
import math

import numpy as np
import pytest

from paper_1610_07522_gb300 import inputs as IN


def test_workload_sizes():
    W = IN.WORKLOADS
    assert (W["sly4_16cubed_16n16p_fp64"].grid, W["sly4_16cubed_16n16p_fp64"].N,
            W["sly4_16cubed_16n16p_fp64"].Z) == ((16, 16, 16), 16, 16)
    w = W["sly4_24cubed_280n120p_coulomb_fp64"]
    assert (w.grid, w.N, w.Z, w.coulomb) == ((24, 24, 24), 280, 120, True)
    w = W["sly4_32cubed_700n300p"]
    assert (w.grid, w.N, w.Z) == ((32, 32, 32), 700, 300)
    w = W["sly4_64cubed_5600n2400p"]
    assert (w.grid, w.N, w.Z) == ((64, 64, 64), 5600, 2400)
    for k in ("sly4_32cubed_3000n3000p", "sly4_48cubed_3000n3000p"):
        assert W[k].N + W[k].Z == 6000
    for w in W.values():
        assert w.x0 == 0.45 and w.E0 == 100.0 and w.dx == (1.0, 1.0, 1.0)


def test_batched_boxes():
    ws = IN.batched_workloads(64)
    assert len(ws) == 64
    want = {16: (86, 37), 20: (168, 72), 24: (290, 125)}
    for i, w in enumerate(ws):
        n = (16, 20, 24)[i % 3]
        assert w.grid == (n, n, n)
        A = round(0.03 * n ** 3)
        assert (w.N + w.Z, w.Z) == (A, math.floor(0.3 * A + 0.5)) and (w.N, w.Z) == want[n]
        assert all(-math.pi <= t < math.pi for t in w.twist)
    assert len({w.twist for w in ws}) == 64 and len({w.seed for w in ws}) == 64
    assert [w.twist for w in IN.batched_workloads(64)] == [w.twist for w in ws]   # seeded


def test_plane_wave_shells():
    labels = IN.plane_wave_labels((16, 16, 16), (1.0, 1.0, 1.0), 200)
    m2 = [mx * mx + my * my + mz * mz for mx, my, mz, _ in labels]
    assert m2 == sorted(m2)
    # spin-degenerate cumulative shell fillings of a cubic box
    counts = [sum(1 for v in m2 if v <= r) for r in range(6)]
    assert counts == [2, 14, 38, 54, 66, 114]
    assert [s for *_, s in labels[:4]] == [0, 1, 0, 1]          # spin up before down
    first = [(mx, my, mz) for mx, my, mz, s in labels[2:14:2]]
    assert first == sorted(first)                               # lexicographic within a shell
    psi = IN.plane_wave_states((8, 8, 8), (1.0, 1.0, 1.0), IN.plane_wave_labels((8, 8, 8), (1.0, 1.0, 1.0), 20))
    S = np.einsum("aszyx,bszyx->ab", np.conj(psi), psi)         # dx^3 = 1
    assert np.max(np.abs(S - np.eye(20))) < 1e-12


@pytest.mark.parametrize("init", ["blobs", "pasta_sphere", "pasta_rod", "pasta_slab"])
def test_starting_densities(init):
    w = IN.Workload(name="t", grid=(16, 16, 16), dx=(1.0, 1.0, 1.0), N=30, Z=12, init=init, seed=5)
    inp = IN.make_inputs(w)
    rho, tau = inp["rho0"], inp["tau0"]
    assert rho.shape == (2, 16, 16, 16) and np.all(rho > 0)
    assert abs(rho[0].sum() - 30) < 1e-10 and abs(rho[1].sum() - 12) < 1e-10
    assert np.allclose(tau, 0.6 * (3 * np.pi ** 2) ** (2 / 3) * rho ** (5 / 3))
    assert len(inp["psi0"]) == 2 and inp["psi0"][0].shape == (30, 2, 16, 16, 16)
    again = IN.make_inputs(w)
    assert np.array_equal(again["psi0"][1], inp["psi0"][1])
    if init == "pasta_slab":                                    # uniform in x and y
        assert np.allclose(rho[0], rho[0][:, :1, :1])
    if init == "pasta_rod":                                     # uniform along z
        assert np.allclose(rho[0], rho[0][:1])
    if init == "pasta_sphere":                                  # densest at the centre
        assert rho[0][8, 8, 8] == rho[0].max()
