"""Pins of the learned-damping oracle (oracle/precond_oracle.py) against
things it does not compute itself: brute-force loops, lattice symmetry,
central finite differences and closed forms."""
import numpy as np
import pytest

from oracle import precond_oracle as P
from oracle import sky_oracle as O


def _rand_theta(rng, scale=0.3):
    return scale * rng.standard_normal(P.NPARAM)


def test_parameter_count():
    assert P.NPARAM == 16 * 3 * 27 + 16 + 16 * 16 * 27 + 16 + 16 * 27 + 1 == 8673


def test_conv_matches_brute_force_loop():
    rng = np.random.default_rng(11)
    nz, ny, nx = 3, 4, 5
    x = rng.standard_normal((2, nz, ny, nx))
    Wt = rng.standard_normal((3, 2, 27))
    b = rng.standard_normal(3)
    out = P.conv(x, Wt, b)
    ref = np.zeros_like(out)
    for o in range(3):
        for z in range(nz):
            for y in range(ny):
                for xx in range(nx):
                    s = b[o]
                    for i in range(2):
                        for dz in (-1, 0, 1):
                            for dy in (-1, 0, 1):
                                for dx in (-1, 0, 1):
                                    t = 9 * (dz + 1) + 3 * (dy + 1) + dx + 1
                                    s += Wt[o, i, t] * x[i, (z + dz) % nz, (y + dy) % ny, (xx + dx) % nx]
                    ref[o, z, y, xx] = s
    assert np.max(np.abs(out - ref)) < 1e-12


def test_one_hot_kernel_is_a_shift():
    rng = np.random.default_rng(12)
    x = rng.standard_normal((1, 4, 5, 6))
    Wt = np.zeros((1, 1, 27))
    Wt[0, 0, 9 * 2 + 3 * 0 + 1] = 1.0          # d = (dz, dy, dx) = (1, -1, 0)
    out = P.conv(x, Wt, np.zeros(1))[0]
    for z in range(4):
        for y in range(5):
            for xx in range(6):
                assert out[z, y, xx] == x[0, (z + 1) % 4, (y - 1) % 5, xx]


def test_forward_translation_equivariant():
    rng = np.random.default_rng(13)
    x = rng.standard_normal((3, 6, 5, 4))
    th = _rand_theta(rng)
    w, _ = P.forward(th, x)
    ws, _ = P.forward(th, np.roll(x, (2, -1, 3), axis=(1, 2, 3)))
    assert np.max(np.abs(ws - np.roll(w, (2, -1, 3), axis=(0, 1, 2)))) < 1e-12
    assert np.all((w > 0) & (w < P.WMAX))


def test_zero_last_layer_gives_constant_weight():
    rng = np.random.default_rng(14)
    parts = P.unpack(_rand_theta(rng))
    parts["W3"][:] = 0.0
    parts["b3"][:] = -np.log(P.WMAX - 1.0)
    w, _ = P.forward(P.pack(parts), rng.standard_normal((3, 4, 4, 4)))
    assert np.max(np.abs(w - 1.0)) < 1e-14


def _sample(rng, shape=(4, 5, 3)):
    x = rng.standard_normal((3,) + shape)
    a = rng.uniform(0.5, 2.0, shape)
    b = rng.uniform(-1.0, 2.0, shape)
    c = b * b / a + rng.uniform(0.1, 1.0, shape)      # c >= b^2/a: a valid |d - w g|^2
    return x, np.stack([a, b, c])


def test_loss_closed_forms():
    rng = np.random.default_rng(15)
    _, abc = _sample(rng)
    assert P.loss(np.zeros(abc.shape[1:]), abc) == pytest.approx(1.0, abs=1e-15)
    wopt = abc[1] / abc[0]
    lmin = P.loss(wopt, abc)
    assert lmin == pytest.approx(float(np.sum(abc[2] - abc[1] ** 2 / abc[0]) / np.sum(abc[2])), rel=1e-12)
    for _ in range(5):
        assert P.loss(wopt + 0.1 * rng.standard_normal(wopt.shape), abc) > lmin


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(16)
    x, abc = _sample(rng)
    th = _rand_theta(rng, 0.4)
    w, cache = P.forward(th, x)
    g = P.backward(th, w, cache, abc)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in P.SHAPES])
    idx = []
    for k in range(len(P.SHAPES)):
        idx += list(rng.choice(np.arange(offs[k], offs[k + 1]), size=min(6, offs[k + 1] - offs[k]),
                               replace=False))
    h = 1e-6
    for i in idx:
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (P.loss(P.forward(tp, x)[0], abc) - P.loss(P.forward(tm, x)[0], abc)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_input_gradient_matches_central_differences():
    rng = np.random.default_rng(17)
    x = rng.standard_normal((2, 3, 4, 5))
    Wt = rng.standard_normal((3, 2, 27))
    dout = rng.standard_normal((3, 3, 4, 5))
    din = P.conv_input_grad(dout, Wt)
    dW, db = P.conv_weight_grad(dout, x)
    f = lambda xx, WW, bb: float(np.sum(dout * P.conv(xx, WW, bb)))
    b0 = np.zeros(3)
    h = 1e-6
    for _ in range(8):
        i = tuple(rng.integers(0, s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        assert abs((f(xp, Wt, b0) - f(xm, Wt, b0)) / (2 * h) - din[i]) < 1e-6
        j = tuple(rng.integers(0, s) for s in Wt.shape)
        Wp, Wm = Wt.copy(), Wt.copy()
        Wp[j] += h
        Wm[j] -= h
        assert abs((f(x, Wp, b0) - f(x, Wm, b0)) / (2 * h) - dW[j]) < 1e-6
    assert np.allclose(db, dout.sum(axis=(1, 2, 3)))


def test_first_adam_step_is_signed_learning_rate():
    rng = np.random.default_rng(18)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    t1, m, v = P.adam(th, g, np.zeros(50), np.zeros(50), 1, lr=0.01, eps=0.0)
    assert np.allclose(t1, th - 0.01 * np.sign(g), atol=1e-15)
    # constant gradients keep the bias-corrected step at lr
    t2, _, _ = P.adam(t1, g, m, v, 2, lr=0.01, eps=0.0)
    assert np.allclose(t2, t1 - 0.01 * np.sign(g), atol=1e-14)


def _grid_and_states(rng, I=3, n=(4, 4, 4)):
    grid = O.Grid(n, (1.0, 1.0, 1.0))
    psi = rng.standard_normal((I, 2) + grid.shape) + 1j * rng.standard_normal((I, 2) + grid.shape)
    return grid, O.orthonormalize(psi, grid)


def test_weighted_step_reduces_to_plain_and_is_linear():
    rng = np.random.default_rng(19)
    grid, psi = _grid_and_states(rng)
    U = rng.uniform(-40, 0, grid.shape)
    B = 20.7 + rng.uniform(0, 5, grid.shape)
    W = rng.uniform(-2, 2, (3,) + grid.shape)
    hpsi = O.apply_h(psi, U, B, W, grid)
    eps, _ = O.sp_energies(psi, hpsi, grid)
    phi = O.damped_step(psi, hpsi, eps, grid, 20.7, 0.45, 100.0)
    assert np.max(np.abs(P.weighted_damped_step(psi, phi, np.ones(grid.shape)) - phi)) < 1e-15
    # x0 enters Eq. dampstep linearly: a constant w = 2 is the step with 2 x0
    phi2 = O.damped_step(psi, hpsi, eps, grid, 20.7, 0.9, 100.0)
    assert np.max(np.abs(P.weighted_damped_step(psi, phi, 2.0 * np.ones(grid.shape)) - phi2)) < 1e-12


def test_stats_special_cases():
    rng = np.random.default_rng(20)
    grid, psi = _grid_and_states(rng, I=4)
    phi = psi + 0.1 * (rng.standard_normal(psi.shape) + 1j * rng.standard_normal(psi.shape))
    # psi inside the span of psi_star (a unitary mix of it): d = 0
    Q, _ = np.linalg.qr(rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)))
    star = np.einsum("ab,b...->a...", Q, psi)
    abc = P.stats(psi, phi, star, grid.dV)
    assert np.max(np.abs(abc[1:])) < 1e-12
    assert np.allclose(abc[0], np.sum(np.abs(psi - phi) ** 2, axis=(0, 1)))
    # psi orthogonal to psi_star: d = psi, c = the density of psi summed over spin
    r = rng.standard_normal((6, 2) + grid.shape) + 1j * rng.standard_normal((6, 2) + grid.shape)
    R, Pm = r.reshape(6, -1), psi.reshape(4, -1)
    R = R - (Pm.T @ (grid.dV * np.conj(Pm) @ R.T)).T      # remove the psi components
    star2 = O.orthonormalize(R.reshape(r.shape), grid)
    abc2 = P.stats(psi, phi, star2, grid.dV)
    assert np.allclose(abc2[2], np.sum(np.abs(psi) ** 2, axis=(0, 1)), atol=1e-12)
    assert np.allclose(abc2[1], np.sum((np.conj(psi - phi) * psi).real, axis=(0, 1)), atol=1e-12)


def test_weighted_iteration_keeps_the_fixed_point():
    """Eigenstates of a frozen h are a fixed point of the step for every w:
    the weighted iteration returns the same Ritz values and the same span."""
    rng = np.random.default_rng(21)
    grid = O.Grid((4, 4, 4), (1.0, 1.0, 1.0))
    p = dict(t0=-2488.91, t1=486.82, t2=-546.39, t3=13777.0, x0=0.834, x1=-0.344, x2=-1.0,
             x3=1.354, alpha=1.0 / 6.0, W0=123.0, hb2m_n=20.73553, hb2m_p=20.73553, e2=1.43996)
    U = np.stack([rng.uniform(-40, 0, grid.shape) for _ in range(2)])
    Bf = np.stack([20.7 + rng.uniform(0, 3, grid.shape) for _ in range(2)])
    Wf = np.stack([rng.uniform(-1, 1, (3,) + grid.shape) for _ in range(2)])
    psi = []
    for q in range(2):
        Hd = O.dense_h(U[q], Bf[q], Wf[q], grid) * grid.dV
        lam, vec = np.linalg.eigh(0.5 * (Hd + Hd.conj().T) / grid.dV)
        psi.append((vec[:, :3].T / np.sqrt(grid.dV)).reshape((3, 2) + grid.shape))
    st = O.State(psi, U, Bf, Wf)
    ref = [x.copy() for x in psi]
    w_of = lambda q, U_, B_, W_: rng.uniform(0.2, 3.5, grid.shape)
    rec = O.iterate(st, grid, p, False, 0.45, 100.0, frozen=True, damping=w_of)
    for q in range(2):
        Hd = O.dense_h(U[q], Bf[q], Wf[q], grid)
        lam = np.linalg.eigvalsh(0.5 * (Hd + Hd.conj().T))[:3]
        assert np.max(np.abs(rec["lam"][q] - lam)) < 1e-9
        ov = grid.dV * np.conj(ref[q].reshape(3, -1)) @ st.psi[q].reshape(3, -1).T
        assert np.max(np.abs(np.abs(np.linalg.svd(ov, compute_uv=False)) - 1.0)) < 1e-9
