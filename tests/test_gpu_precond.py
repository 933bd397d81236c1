"""Parity of the learned-damping entry points with the FP64 CPU oracle (GPU).

The network runs in FP32 on the GPU and in FP64 in the oracle.  Tolerances
follow from FP32 rounding: w lies in (0, 4) and is formed from sums of
27 x 16 products of O(1) terms, so its error is a few 1e-6; gradients are
compared against the largest component (1e-4), the loss within 1e-5
relative.  The weighted step, the cross overlap and the statistics are FP64
on both sides (1e-12 of the largest magnitude).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from oracle import precond_oracle as PO
from paper_1610_07522_gb300 import binding as B
from paper_1610_07522_gb300 import inputs as IN

pytestmark = pytest.mark.gpu

P = dict(IN.SLY4)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def maxrel(got, want):
    return float(np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300))


class Ctx:
    def __init__(self, grid, prec=B.SKY_F64, max_states=64, twist=(0.0, 0.0, 0.0)):
        self.grid = O.Grid(grid, (1.0, 1.0, 1.0), twist)
        self.ctx = B.sky_init(grid, (1.0, 1.0, 1.0), P, False, twist, prec, max_states,
                              torch.cuda.current_stream().cuda_stream)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        B.sky_sync(self.ctx)
        B.sky_destroy(self.ctx)


def _fields(n, rng):
    U = IN.random_smooth_field(n, rng, -40.0, 30.0)
    Bf = IN.random_smooth_field(n, rng, 24.0, 5.0)
    W = np.stack([IN.random_smooth_field(n, rng, 0.0, 4.0) for _ in range(3)])
    return U, Bf, W


def _abc(shape, rng):
    a = rng.uniform(0.5, 2.0, shape)
    b = rng.uniform(-1.0, 3.0, shape)
    c = b * b / a + rng.uniform(0.1, 1.0, shape)
    return np.stack([a, b, c])


GRIDS = [(16, 16, 16), (12, 16, 20), (8, 24, 12)]


@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("q", [0, 1])
def test_net_forward_loss_and_gradient(grid, q):
    rng = np.random.default_rng(100 + sum(grid) + q)
    with Ctx(grid) as c:
        g = c.grid
        U, Bf, W = _fields(g.n, rng)
        theta = (0.3 * rng.standard_normal(PO.NPARAM)).astype(np.float32)
        abc = _abc(g.shape, rng)
        x = PO.features(U, Bf, W, P["hb2m_n"] if q == 0 else P["hb2m_p"])
        w_want, cache = PO.forward(theta.astype(np.float64), x)
        l_want = PO.loss(w_want, abc)
        g_want = PO.backward(theta.astype(np.float64), w_want, cache, abc)
        G = g.G
        d_th = dev(theta)
        ws = torch.zeros(B.SKY_NET_WS_PER_POINT * G, dtype=torch.float32, device="cuda:0")
        w = torch.zeros(G, dtype=torch.float32, device="cuda:0")
        d_abc, norm = dev(abc.reshape(3, -1)), dev(np.array([abc[2].sum()]))
        grad = torch.zeros(PO.NPARAM, dtype=torch.float64, device="cuda:0")
        loss = torch.zeros(1, dtype=torch.float64, device="cuda:0")
        B.sky_net_forward(c.ctx, q, d_th, dev(U), dev(Bf), dev(W), ws, w)
        B.sky_net_backward(c.ctx, d_th, ws, d_abc, norm, grad, loss)
        w_got = host(w).reshape(g.shape)
        assert np.max(np.abs(w_got - w_want)) < 2e-5
        assert abs(host(loss)[0] - l_want) < 1e-5 * abs(l_want)
        gg = host(grad)
        assert maxrel(gg, g_want) < 1e-4
        # per block of parameters as well, so a wrong small block cannot hide
        o = 0
        for name, shape in PO.SHAPES:
            n = int(np.prod(shape))
            blk_w, blk_g = g_want[o:o + n], gg[o:o + n]
            assert np.max(np.abs(blk_g - blk_w)) < 1e-4 * max(np.max(np.abs(blk_w)), 1e-3 * np.max(np.abs(g_want))), name
            o += n
        # a scaled forward moves the step's weight toward 1 and keeps the
        # network's own weight for training: a second backward accumulates
        B.sky_net_forward(c.ctx, q, d_th, dev(U), dev(Bf), dev(W), ws, w, 0.25)
        assert np.max(np.abs(host(w).reshape(g.shape) - (1.0 + 0.25 * (w_want - 1.0)))) < 1e-5
        B.sky_net_backward(c.ctx, d_th, ws, d_abc, norm, grad, loss)
        assert maxrel(host(grad), 2 * g_want) < 1e-4
        assert abs(host(loss)[0] - 2 * l_want) < 2e-5 * abs(l_want)


def test_untrained_net_is_the_plain_step():
    from paper_1610_07522_gb300 import learned
    rng = np.random.default_rng(7)
    with Ctx((16, 12, 8)) as c:
        U, Bf, W = _fields(c.grid.n, rng)
        th = dev(learned.init_params(3))
        ws = torch.zeros(B.SKY_NET_WS_PER_POINT * c.grid.G, dtype=torch.float32, device="cuda:0")
        w = torch.zeros(c.grid.G, dtype=torch.float32, device="cuda:0")
        B.sky_net_forward(c.ctx, 0, th, dev(U), dev(Bf), dev(W), ws, w)
        assert np.max(np.abs(host(w) - 1.0)) < 1e-6


def test_adam_matches_oracle():
    rng = np.random.default_rng(8)
    with Ctx((8, 8, 8)) as c:
        theta = rng.standard_normal(PO.NPARAM).astype(np.float32)
        th_o = theta.astype(np.float64)
        m_o, v_o = np.zeros(PO.NPARAM), np.zeros(PO.NPARAM)
        d_th = dev(theta)
        grad = torch.zeros(PO.NPARAM, dtype=torch.float64, device="cuda:0")
        m = torch.zeros_like(grad)
        v = torch.zeros_like(grad)
        for step in range(1, 5):
            gvec = rng.standard_normal(PO.NPARAM) * 10.0 ** rng.uniform(-3, 1)
            grad.copy_(dev(gvec))
            B.sky_net_adam(c.ctx, d_th, grad, m, v, step, 1e-2, 0.9, 0.999, 1e-8)
            th_o, m_o, v_o = PO.adam(th_o, gvec, m_o, v_o, step, 1e-2, 0.9, 0.999, 1e-8)
            th_o = th_o.astype(np.float32).astype(np.float64)   # the device stores theta in FP32
        assert np.max(np.abs(host(d_th) - th_o)) < 1e-6
        assert maxrel(host(m), m_o) < 1e-12 and maxrel(host(v), v_o) < 1e-12
        assert np.all(host(grad) == 0.0)


@pytest.mark.parametrize("prec", [B.SKY_F64, B.SKY_F32])
def test_weighted_damped_step(prec):
    rng = np.random.default_rng(9)
    with Ctx((12, 16, 20), prec=prec, twist=(0.4, -1.0, 2.2)) as c:
        g = c.grid
        I = 7
        psi = IN.random_spinors(g.n, I, rng)
        hpsi = IN.random_spinors(g.n, I, rng) * 20.0
        eps = rng.uniform(-40, 10, I)
        wv = rng.uniform(0.2, 3.5, g.shape)
        plain = O.damped_step(psi, hpsi, eps, g, P["hb2m_p"], 0.45, 100.0)
        want = PO.weighted_damped_step(psi, plain, wv)
        cd = torch.complex128 if prec == B.SKY_F64 else torch.complex64
        d_psi, d_h = dev(psi).to(cd), dev(hpsi).to(cd)
        phi = torch.zeros_like(d_psi)
        B.sky_damped_step(c.ctx, 1, d_psi, d_h, dev(eps), phi, I, 0.45, 100.0,
                          dev(wv.astype(np.float32)))
        tol = 1e-12 if prec == B.SKY_F64 else 5e-6
        # the oracle's weight is the same FP32 value the device reads
        want32 = PO.weighted_damped_step(psi, plain, wv.astype(np.float32).astype(np.float64))
        assert maxrel(host(phi), want32) < tol
        assert maxrel(host(phi), want) < 1e-6


@pytest.mark.parametrize("prec", [B.SKY_F64, B.SKY_F32, B.SKY_F32_BF16X3])
@pytest.mark.parametrize("I", [1, 40, 70])
def test_cross_overlap_and_stats(prec, I):
    rng = np.random.default_rng(10 + I)
    with Ctx((12, 16, 20), prec=prec, max_states=80) as c:
        g = c.grid
        psi = IN.random_spinors(g.n, I, rng)
        star = O.orthonormalize(IN.random_spinors(g.n, I, rng) + 0.5 * psi, g)
        phi = psi + 0.05 * IN.random_spinors(g.n, I, rng)
        cd = torch.complex128 if prec == B.SKY_F64 else torch.complex64
        if prec != B.SKY_F64:   # both sides see the FP32-rounded states
            psi, star, phi = (a.astype(np.complex64).astype(np.complex128) for a in (psi, star, phi))
        X_want = g.dV * (np.conj(star.reshape(I, -1)) @ psi.reshape(I, -1).T)
        d_psi, d_star, d_phi = dev(psi).to(cd), dev(star).to(cd), dev(phi).to(cd)
        X = torch.zeros((I, I), dtype=torch.complex128, device="cuda:0")
        B.sky_cross_overlap(c.ctx, d_star, d_psi, I, X)
        assert maxrel(host(X), X_want) < 1e-12
        # stats on the device's own projection, then against the oracle's statistics
        pp = torch.zeros_like(d_psi)
        B.sky_rotate(c.ctx, d_star, X, I, pp)
        abc = torch.zeros((3, g.G), dtype=torch.float64, device="cuda:0")
        norm = torch.zeros(1, dtype=torch.float64, device="cuda:0")
        B.sky_precond_stats(c.ctx, d_psi, d_phi, pp, I, abc, norm)
        want = PO.stats(psi, phi, star, g.dV).reshape(3, -1)
        tol = {B.SKY_F64: 1e-11, B.SKY_F32: 2e-5, B.SKY_F32_BF16X3: 2e-4}[prec]
        got = host(abc)
        for k in range(3):
            assert maxrel(got[k], want[k]) < tol, k
        assert abs(host(norm)[0] - got[2].sum()) < 1e-12 * got[2].sum()


def test_learned_iterations_match_oracle():
    """Three iterations of the 8^3, 4n+4p workload with a fixed random network:
    the device path (FP32 network, FP64 spinors) against the oracle iteration
    with the FP64 network.  The FP32 weight enters the update linearly
    (|dw| ~ 1e-6), so energies agree to ~1e-7 relative."""
    from paper_1610_07522_gb300 import learned
    from paper_1610_07522_gb300.solver import Solver
    w = IN.WORKLOADS["sly4_8cubed_4n4p"]
    inp = IN.make_inputs(w)
    rng = np.random.default_rng(12)
    theta = learned.init_params(5)
    parts = PO.unpack(theta.astype(np.float64).copy())
    parts["W3"][:] = 0.2 * rng.standard_normal(parts["W3"].shape)
    theta = PO.pack(parts).astype(np.float32)
    g = O.Grid(w.grid, w.dx, w.twist)
    hb2m = (w.params["hb2m_n"], w.params["hb2m_p"])
    damping = lambda q, U, Bq, Wq: PO.forward(theta.astype(np.float64), PO.features(U, Bq, Wq, hb2m[q]))[0]
    st = O.initial_state(inp["psi0"], g, w.params, w.coulomb)
    recs = [O.iterate(st, g, w.params, w.coulomb, w.x0, w.E0, damping=damping) for _ in range(3)]
    s = Solver(w, prec=B.SKY_F64)
    s.set_damping(learned.DampingNet("cuda:0", theta=theta))
    s.load(inp["psi0"])
    for k in range(3):
        s.step()
        E, de, _ = s.energy()
        assert abs(E - recs[k]["E"]) < 1e-6 * abs(recs[k]["E"]) + 1e-9
        lam = host(s.lam)
        want = np.concatenate(recs[k]["lam"])
        assert np.max(np.abs(lam - want)) < 1e-5
    # the weight was not 1: the same run without it differs
    s2 = Solver(w, prec=B.SKY_F64)
    s2.load(inp["psi0"])
    for _ in range(3):
        s2.step()
    assert abs(s2.energy()[0] - recs[2]["E"]) > 1e-5
    s.close()
    s2.close()
