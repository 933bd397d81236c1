"""The device-side generator of noisy plane waves (used for the 64^3,
5600 n + 2400 p workload) follows the recipe of the NumPy generator: state a
is its plane wave e^{i k.r}/sqrt(L^3) in its spin component plus complex
noise of variance amp^2 / L^3 per voxel and component (checked on the CPU
device: the projection on the plane wave and the residual's variance)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1610_07522_gb300 import inputs as IN


def test_device_noisy_plane_waves_follow_the_recipe():
    grid, dx, I, amp = (16, 16, 16), (1.0, 1.0, 1.0), 40, 0.1
    psi = IN.noisy_plane_waves_device(grid, dx, I, amp, 7, "cpu", torch.complex128).numpy()
    pw = IN.plane_wave_states(grid, dx, IN.plane_wave_labels(grid, dx, I))
    vol = 16.0 ** 3
    G = 16 ** 3
    res = psi - pw
    var = np.mean(np.abs(res) ** 2)
    assert abs(var - amp ** 2 / vol) < 0.05 * amp ** 2 / vol
    # every state is dominated by its own plane wave (noise projection ~ amp / sqrt(2 G))
    proj = np.einsum("aszyx,aszyx->a", np.conj(pw), psi)
    assert np.max(np.abs(proj - 1.0)) < 6 * amp / math.sqrt(2 * G)
    # seeded: the same seed gives the same states
    again = IN.noisy_plane_waves_device(grid, dx, I, amp, 7, "cpu", torch.complex128).numpy()
    assert np.array_equal(psi, again)
